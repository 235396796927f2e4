/*
 * g6gb.h -- GRAPE-6-style direct-summation force library for GB300 (sm_103a).
 *
 * Method: Gaburov, Harfst & Portegies Zwart, "SAPPORO: A way to turn your
 * graphics cards into a GRAPE-6" (arXiv:0902.4463).  The library evaluates
 * the data-parallel hot path of a 4th-order Hermite block-time-step N-body
 * integrator (Sect. 2): it predicts every j-particle to the block time
 * (Sect. 2.2, Eq. 1 and Eq. 2), then for each active i-particle sums the
 * softened acceleration, jerk and potential over all j-particles and finds the
 * nearest neighbour and, optionally, the neighbour list (Sect. 2.3, 2.5, 4).
 *
 * Precision (Sect. 2.2, 2.3): bulk pair arithmetic in FP32; positions are
 * double-single (hi + lo floats) and separations use the simplified DS
 * difference of Eq. 3; predicted positions come from the DS + SP addition of
 * Sect. 2.2 (or, with G6X_PREC_DS_X64, from an FP64 addition split into DS);
 * partial sums are carried as compensated FP32 pairs and reduced in FP64.
 * g6x_set_precision(cid, G6X_PREC_FP64) selects an all-FP64 path instead.
 *
 * Units: G = 1.  pot is the negative physical potential, -sum m_j/sqrt(r^2+eps2).
 * Self-interaction is excluded by index: the j-particle whose `index` equals
 * the i-particle's index does not act on it.  Indices must be >= 0.
 *
 * Host threads: the library's host loops over large blocks (i-record and
 * j-record staging, sorting, copies of results, the drivers' prediction and
 * correction, per-cluster batch work) run on one process-wide pool of
 * G6GB_HOST_THREADS threads (default min(cores, 16)), started on first use;
 * a loop that finds the pool busy (another caller) runs on its own thread.
 *
 * Calling sequence (Sect. 2.1, Sect. 2.5; the same order as GRAPE-6):
 *   g6_open(cid);
 *   per block step:  g6_set_j_particle(...) for each particle corrected last
 *                    step; g6_set_ti(cid, t_blk);
 *                    g6calc_firsthalf(...); g6calc_lasthalf(...) [or 2];
 *                    optionally g6_read_neighbour_list / g6_get_neighbour_list;
 *   g6_close(cid);
 *
 * Ownership: every array argument is owned by the caller.  g6_set_j_particle
 * and g6calc_firsthalf copy what they need before returning, so the caller may
 * reuse its arrays at once.  g6calc_lasthalf writes into the caller's arrays.
 *
 * Errors: functions return 0 on success or a negative G6_E* code.
 * g6calc_firsthalf returns void (as in GRAPE-6): its error is latched and
 * returned by the next g6calc_lasthalf.  A context is not thread-safe; use one
 * context (cluster id) per thread.  Nothing in this library traps or aborts.
 */
#ifndef G6GB_H
#define G6GB_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---------------------------------------------------------------- limits */
#define G6_MAX_CLUSTERS   16     /* cluster ids 0 .. 15                          */
#define G6_NPIPES_DEFAULT 256    /* i-particles per call (Sect. 2.5 footnote)    */
#define G6_MAXNB          256    /* neighbour-list length (Sect. 4)              */
#define G6_NJ_DEFAULT     (1 << 21) /* default j-memory capacity of g6_open      */

/* ----------------------------------------------------------- error codes */
#define G6_OK          0
#define G6_EINVAL    (-22)  /* bad argument: cluster id, address, count, eps2 */
#define G6_ENOTOPEN  (-19)  /* cluster id not open                            */
#define G6_EBUSY     (-16)  /* cluster id already open / call out of order    */
#define G6_ENOMEM    (-12)  /* device or pinned host allocation failed        */
#define G6_EIO        (-5)  /* CUDA runtime error                             */
#define G6_ETIMEDOUT (-110) /* a device-side bounded wait gave up             */
#define G6_ENODEV    (-6)   /* no CUDA device / library built for another GPU */
#define G6_EOVERFLOW  (1)   /* g6_read_neighbour_list: some list overflowed   */

/* ------------------------------------------------ GRAPE-6 compatible API */

/* Allocate a context for cluster id `clusterid` on the current CUDA device,
 * with room for G6_NJ_DEFAULT j-particles (env G6GB_NJ overrides) and
 * g6_npipes() i-particles per call.  Returns 0 or G6_EINVAL / G6_EBUSY /
 * G6_ENOMEM / G6_EIO / G6_ENODEV. */
int g6_open(int clusterid);

/* Free everything the context owns.  Returns 0 or G6_EINVAL / G6_ENOTOPEN. */
int g6_close(int clusterid);

/* Maximum i-particles per g6calc call: 256 (Sect. 2.5 footnote), or the
 * value of env G6GB_NPIPES when set. */
int g6_npipes(void);

/* GRAPE-6 fixed-point scale settings.  This library works in floating point,
 * so both are accepted and ignored.  Return 0. */
int g6_set_tunit(int newtunit);
int g6_set_xunit(int newxunit);

/* Set the block time t_blk to which the j-particles are predicted by the
 * next g6calc_firsthalf (Sect. 2.2).  Cheap; marks the prediction stale. */
int g6_set_ti(int clusterid, double ti);

/* Store one j-particle in j-memory slot `address` (0 <= address < capacity)
 * (Sect. 2.1: only corrected particles are sent each step).
 *   index : particle id (>= 0) used for self-exclusion and returned by the
 *           nearest-neighbour and neighbour-list calls;
 *   tj    : time of this state; prediction uses dt = t_blk - tj (Sect. 2.2);
 *   dtj   : the particle's own step (accepted, unused);
 *   mass  : m_j;
 *   k18   : snap / 18 (accepted, ignored: the predictor is 3rd order, Eq. 1);
 *   j6    : jerk / 6;   a2: acceleration / 2 (pre-scaled Taylor terms);
 *   v, x  : velocity and position at tj.
 * The record is staged on the host and uploaded by the next firsthalf.
 * Returns 0 or G6_EINVAL / G6_ENOTOPEN / G6_ENOMEM. */
int g6_set_j_particle(int clusterid, int address, int index, double tj,
                      double dtj, double mass, const double k18[3],
                      const double j6[3], const double a2[3],
                      const double v[3], const double x[3]);

/* Start the force on ni i-particles (ni <= the context's ni_max, default
 * g6_npipes()) from j-slots 0 .. nj-1 (Sect. 2.3).  xi, vi are the
 * i-particles' predicted FP64 state at t_blk (the host predicts i-particles,
 * Sect. 2.1); index[] their ids; eps2 >= 0 the softening of this i-block
 * (Sect. 2.5); h2[] (may be NULL) the squared neighbour radius per i.  aold,
 * j6old, phiold are accepted and ignored (no fixed-point scaling is needed).
 * Asynchronous: uploads pending j updates and the i-data, predicts the
 * j-particles if t_blk or j-memory changed, launches the force and the
 * reduction, and starts the copy back.  Errors are latched for lasthalf. */
void g6calc_firsthalf(int clusterid, int nj, int ni, const int index[],
                      const double xi[][3], const double vi[][3],
                      const double aold[][3], const double j6old[][3],
                      const double phiold[], double eps2, const double h2[]);

/* Wait for the force started by firsthalf and write acc, jerk, pot (ni
 * entries each).  The argument list repeats firsthalf's as in GRAPE-6; nj,
 * ni and index must match.  Returns 0, the latched firsthalf error, or
 * G6_EIO / G6_ETIMEDOUT. */
int g6calc_lasthalf(int clusterid, int nj, int ni, const int index[],
                    const double xi[][3], const double vi[][3], double eps2,
                    const double h2[], double acc[][3], double jerk[][3],
                    double pot[]);

/* As g6calc_lasthalf, plus nnbindex[i] = index of the nearest j-particle
 * (smallest unsoftened |r|^2, ties to the lower j-slot), or -1 if none
 * (Sect. 2.5). */
int g6calc_lasthalf2(int clusterid, int nj, int ni, const int index[],
                     const double xi[][3], const double vi[][3], double eps2,
                     const double h2[], double acc[][3], double jerk[][3],
                     double pot[], int nnbindex[]);

/* Make the neighbour lists of the last calculation readable on the host
 * (Sect. 4): for each i the j-particles with unsoftened |r|^2 < h2[i],
 * excluding itself, in ascending j-slot order, at most the context's list
 * length of them (G6_MAXNB unless g6x_set_max_neighbours chose another).
 * Synchronous.  The reduction writes the lists straight into pinned host
 * memory, so no copy is made here.  The force kernel keeps each CTA's part
 * of a list in a slot with room for a few entries, grown as lists grow: when
 * a part had more entries than its slot held, this call computes that
 * calculation's lists once more with larger slots (the j-memory must not
 * have changed since: G6_EBUSY), so the lists returned are always complete.  Returns 0, G6_EOVERFLOW (1) if some
 * list was longer than the list length (it is truncated), or a negative
 * error.  Lists exist only if firsthalf got h2 != NULL (or g6x_calc_dev
 * nl != 0, whose d_irec must then stay unchanged until this call). */
int g6_read_neighbour_list(int clusterid);

/* Neighbour list of i-particle number ipipe (0 <= ipipe < ni) of the last
 * calculation: *nblen = list length, nbl[0 .. min(*nblen, maxlength)-1] =
 * particle indices.  Returns 0, G6_EOVERFLOW if *nblen > maxlength or the
 * list overflowed the list length, or a negative error. */
int g6_get_neighbour_list(int clusterid, int ipipe, int maxlength, int *nblen,
                          int nbl[]);

/* ------------------------------------------------------------ extensions */

/* Neighbour-list length of the context, 1 .. G6X_MAXNB_LIMIT entries per
 * i-particle (default G6_MAXNB = 256, the paper's choice, Sect. 4; the paper
 * fixes it at compile time, here it is a setting).  Longer lists cost more
 * pinned host memory (block size x length x 4 B); the force kernel's cost
 * depends on the number of entries found, not on this length.  Applies to later calculations;
 * lists already computed are dropped.  Returns 0 or G6_EINVAL. */
#define G6X_MAXNB_LIMIT 4096
int g6x_set_max_neighbours(int clusterid, int maxnb);
/* The context's list length, or a negative error. */
int g6x_max_neighbours(int clusterid);
/* How often g6_read_neighbour_list computed lists again because a list
 * part outgrew its slot (see there), or a negative error. */
long long g6x_list_reruns(int clusterid);

#define G6X_PREC_DS     0 /* FP32 force with DS separations (Eq. 3) and the
                             DS + SP predictor of Sect. 2.2 (default)       */
#define G6X_PREC_FP64   1 /* all-FP64 prediction and force                 */
#define G6X_PREC_DS_X64 2 /* as G6X_PREC_DS, but predicted positions are
                             formed in FP64 and then split into DS           */
#define G6X_PREC_DS_DSSUB 3 /* as G6X_PREC_DS, but each separation by the full
                             DS subtraction (TwoSum of the high parts, low
                             parts added, one rounding: 9 FP32 operations
                             instead of Eq. 3's 3), an accuracy ablation
                             (Sect. 2.3); neighbour lists and the autotuner
                             use the G6X_PREC_DS kernels                    */

/* As g6_open with an explicit j capacity and i-per-call limit. */
int g6x_open_ex(int clusterid, int nj_max, int ni_max);

/* Select the arithmetic of later calculations (G6X_PREC_*). */
int g6x_set_precision(int clusterid, int mode);

/* Raise (or lower) the i-per-call limit above g6_npipes(). */
int g6x_set_ni_max(int clusterid, int ni_max);

/* Run the context's work on this cudaStream_t (NULL: the context's own
 * stream).  The stream is borrowed, not owned. */
int g6x_set_stream(int clusterid, void *stream);

/* Device allocator hook used by every later g6_open (NULL, NULL: plain
 * cudaMalloc / cudaFree).  alloc(bytes, user) returns a device pointer or
 * NULL; release(ptr, user) frees it. */
typedef void *(*g6x_alloc_fn)(size_t bytes, void *user);
typedef void (*g6x_free_fn)(void *ptr, void *user);
int g6x_set_allocator(g6x_alloc_fn alloc, g6x_free_fn release, void *user);

/* Bulk form of g6_set_j_particle for n particles (arrays of n entries;
 * j6, a2, v, x are n x 3).  Calls with fewer than 8192 particles stop at
 * the first error and return it; larger ones check every entry before
 * staging any (and fill the records on host threads). */
int g6x_set_j_particles(int clusterid, int n, const int address[],
                        const int index[], const double tj[],
                        const double mass[], const double j6[][3],
                        const double a2[][3], const double v[][3],
                        const double x[][3]);

/* Human-readable text for a G6_E* code (static storage). */
const char *g6x_strerror(int code);

/* --------------------------------------- device-resident entry points --
 * The same work on records already in device memory (caller-owned device
 * pointers), asynchronous on the context's stream, no host copies. */

/* One j-particle update, 120 bytes, same meaning as g6_set_j_particle. */
typedef struct {
    double x[3], v[3], a2[3], j6[3];
    double mass, tj;
    int address, index;
} g6x_jrec;

/* One i-particle, 64 bytes: predicted FP64 state, squared neighbour radius
 * (<= 0: no list entries) and id. */
typedef struct {
    double x[3], v[3];
    double h2;
    int index, pad;
} g6x_irec;

/* One result, 64 bytes: acceleration, jerk, potential, nearest-neighbour
 * index (-1 if none) and its unsoftened |r|^2 as computed by the kernel. */
typedef struct {
    double acc[3], jerk[3];
    double pot;
    int nnb;
    float nnr2;
} g6x_out;

/* Scatter n device-resident j records into j-memory (the j-store update). */
int g6x_set_j_dev(int clusterid, int n, const g6x_jrec *d_rec);

/* Predict j-slots 0 .. nj-1 to time ti if stale (Eq. 1, Eq. 2), then force
 * on ni device-resident i records and reduce into ni device-resident
 * results.  nl != 0 also builds neighbour lists (read back with
 * g6_read_neighbour_list).  Returns 0 or a negative error; completion is
 * ordered on the context's stream. */
int g6x_calc_dev(int clusterid, double ti, int nj, int ni,
                 const g6x_irec *d_irec, double eps2, int nl, g6x_out *d_out);

/* Read back the predicted j-particles of the current precision mode for
 * checking: hi[nj][4], lo[nj][4] (DS mode; lo unused in FP64 mode) as float,
 * or x64[nj][4], v64[nj][4] as double.  Pointers may be NULL.  Synchronous. */
int g6x_get_predicted(int clusterid, int nj, float *hi, float *lo, float *vel,
                      double *x64, double *v64);

/* ------------------------------------ allocation-free force entry point --
 * The paper has no counterpart to this call; it exists for callers of this
 * library that must not allocate device memory when they ask for a force:
 * for example an integrator whose device memory belongs to another
 * framework's pool, which forbids cudaMalloc calls outside it, or a
 * latency-critical host loop that cannot accept the device-wide
 * synchronisation that cudaMalloc and cudaFree may cause.  g6x_calc_dev can
 * grow its context's partial-sum buffer when a larger block arrives; this
 * variant never allocates.
 *
 * Same work and arguments as g6x_calc_dev without neighbour lists, except
 * that the partial sums between the force kernel and the reduction live in
 * one fixed device array of G6X_NOALLOC_SCRATCH_BYTES (about 10.1 MiB) that
 * every GPU loading this library holds until the process exits.
 *   - The context must already be open (g6_open allocates, at set-up).
 *   - ni > G6X_NOALLOC_NI_MAX, or a launch whose partial sums cannot fit the
 *     array even on a smaller grid, returns G6_EINVAL before any work.
 *   - The first call on each device looks up the array's device address;
 *     make that first call during set-up, before any stream capture.  The
 *     caller's current device must be the context's (G6_EINVAL otherwise).
 *   - All calls in the process share the array and it keeps the last call's
 *     contents; each call writes every record it reads, so nothing needs
 *     clearing.  Calls that overlap on the GPU (other streams or contexts)
 *     race on the array: issue them one after another.
 * Returns 0 or a negative G6_E* code. */
#define G6X_NOALLOC_NI_MAX        16384
#define G6X_NOALLOC_SCRATCH_BYTES (147456 * 72)
int g6x_calc_dev_noalloc(int clusterid, double ti, int nj, int ni,
                         const g6x_irec *d_irec, double eps2, g6x_out *d_out);

/* Wait for the context's stream and report a device-side error recorded by
 * an earlier g6x_calc_dev (G6_ETIMEDOUT) or a CUDA error.  Returns 0 or the
 * code.  Not allowed between firsthalf and lasthalf (G6_EBUSY). */
int g6x_sync(int clusterid);

/* Pin the force-kernel variant (0 .. variant count - 1; -1: automatic) and
 * the grid size (<= 0: automatic) of later calculations, for tuning. */
int g6x_set_variant(int clusterid, int variant, int grid);

/* Per-kernel CUDA-event timing on the context's stream.  enable != 0 resets
 * the counters and brackets every later launch with events; 0 stops. */
int g6x_set_timing(int clusterid, int enable);

/* Device time (ms, summed) and launch count per phase since timing was
 * enabled: [0] j-memory scatter, [1] predictor, [2] force, [3] reduction.
 * Synchronises the stream.  Either pointer may be NULL. */
int g6x_get_timing(int clusterid, double ms[4], long long count[4]);

/* Autotuner: for each power-of-two block size m = 16 .. m_max (sizes above
 * 2^17 reuse the 2^17 result), time every force-kernel variant of the
 * current precision whose i-tile suits m, on grids of one and two times the
 * resident CTAs, against the nj j-particles in j-memory (i-particles taken
 * from the first m slots), and keep the fastest in a process-wide table that
 * later calculations without a pinned variant use.  Writes the table to
 * `path` when not NULL.  Each candidate is timed as one step: prediction
 * (inside the kernel for the fused-prediction shapes, which take part only
 * with G6X_PREC_DS) + force + reduction.  Synchronous; allocates two
 * scratch buffers.  Returns the number of sizes tuned or a negative error
 * (G6_EINVAL under G6X_PREC_DS_DSSUB, which has no table). */
int g6x_autotune(int clusterid, int nj, int m_max, const char *path);

/* Load a table written by g6x_autotune (g6_open loads the file named by
 * env G6GB_TUNE_FILE once): lines "precision log2(m) variant grid_multiplier"
 * ('#' starts a comment line).  The whole file is checked first; on any bad
 * line nothing changes.  Returns entries read or G6_EINVAL. */
int g6x_load_tuning(const char *path);

/* Forget every tuned entry (back to the built-in choice).  Returns 0. */
int g6x_clear_tuning(void);

/* The launch a calculation of ni i-particles against nj j-particles would
 * get in precision mode `mode` (G6X_PREC_*), with neighbour lists if list
 * != 0, on a GPU of sm_count SMs, from the autotuner's table when it has an
 * entry for this block size and from the built-in choice otherwise; nothing
 * is launched.  out[0..5] = kernel variant, threads along i, threads along
 * j, i-particles per thread, grid size, j-tiles.  The grid counts the
 * resident CTAs per SM of the current device; a host without one gets one
 * CTA per SM.  Not in the paper (it places one block per multiprocessor,
 * Sect. 2.3).  Returns 0 or G6_EINVAL (unknown mode, nj or ni outside
 * 1 .. 2^30, sm_count outside 1 .. 4096, out NULL, lists with
 * G6X_PREC_DS_DSSUB). */
int g6x_plan_launch(int mode, int nj, int ni, int list, int sm_count, int out[6]);

/* The compiled force-kernel variants (the numbers g6x_set_variant, the
 * tuning table and g6x_last_config use).  g6x_variant_info(v, out) fills
 * out[0..7] = threads along i, thread groups along j, i-particles per
 * thread, builds neighbour lists (0/1), precision mode (G6X_PREC_*),
 * predicts its own j-tiles (Eq. 1, Eq. 2 inside the force kernel; 0/1), the
 * variant of the same shape that reads separately predicted tiles (-1 if
 * none), and 1 for the warp-specialised small-block kernel (the whole block
 * is one i-tile of at most threads-along-i x i-per-thread particles; j-store
 * update, prediction, force and reduction in one launch).  Returns the
 * number of variants; g6x_variant_info(-1, NULL) returns it alone.  Needs no
 * GPU.  G6_EINVAL for v outside -1 .. count-1, or out NULL with v >= 0.
 * Not in the paper: these are this library's shapes of the work split of
 * Sect. 2.3. */
int g6x_variant_info(int variant, int out[8]);

/* Launch statistics of the last calculation: kernel variant id, threads
 * along i and j, i-particles per thread, grid size and j-tiles.  Any pointer
 * may be NULL. */
int g6x_last_config(int clusterid, int *variant, int *ti, int *tj, int *ni_per,
                    int *grid, int *jtiles);

/* Limit of each bounded wait of the force kernels for a staged j-tile, in
 * seconds, for every context (default and maximum 2 s; minimum 1e-6).  A
 * wait that runs out makes the kernel record G6_ETIMEDOUT, which the next
 * lasthalf / g6x_sync / g6x_batch_calc returns; the context stays usable.
 * (The wait for the kernel's own copies in flight after a timeout always
 * allows the full 2 s, so no copy lands after the kernel has exited.)
 * Returns 0 or G6_EINVAL. */
int g6x_set_wait_limit(double seconds);

/* Check the timeout path: launch one bounded wait, with the current limit,
 * on an mbarrier that nothing ever completes, on the context's stream, and
 * return what g6x_sync then reports: G6_ETIMEDOUT when the wait ran out and
 * was reported as the force kernels report it (0 would mean it did not). */
int g6x_probe_wait_timeout(int clusterid);

/* Measure the FP32 rate the force kernel's roofline is taken against: on
 * the current device, every SM runs 8 CTAs of 256 threads, each thread 8
 * independent chains of packed FP32x2 fused multiply-adds, iters x 16 per
 * chain; the launch is timed with CUDA events after one short warm-up
 * launch.  *tflops = 4 flop x 16 x 8 x iters x threads / time (TFLOP/s);
 * *ms (may be NULL) = the timed launch.  Not in the paper: the roofline
 * check of the FP32-bound force (Sect. 3.1 counts 60 flop per pair).
 * Allocates and frees its own small buffer, stream and events.  Returns 0,
 * G6_EINVAL (iters outside 1 .. 2^24, tflops NULL), G6_ENODEV, G6_ENOMEM or
 * G6_EIO. */
int g6x_fp32_probe(int iters, double *tflops, double *ms);

/* The FP64 counterpart, the roofline denominator of the all-FP64 force
 * kernel (the comparison kernel of the precision argument, Sect. 2.3): the
 * same launch shape, each thread 8 independent chains of FP64 fused
 * multiply-adds, iters x 16 per chain.  *tflops = 2 flop x 16 x 8 x iters x
 * threads / time.  GB300's FP64 pipe is a small fraction of its FP32 rate,
 * so a few hundred iters already take milliseconds.  Same ownership and
 * returns as g6x_fp32_probe. */
int g6x_fp64_probe(int iters, double *tflops, double *ms);

/* Number of kernels launched on the context's stream since g6_open. */
long long g6x_launch_count(int clusterid);

/* ----------------------------------- Hermite block-time-step driver ----
 * A plain C++ 4th-order Hermite predictor-corrector with power-of-two block
 * time steps (Sect. 2, Sect. 2.1) that drives the g6_* calls above: it
 * predicts the active i-particles on the host, corrects them (Makino &
 * Aarseth 1992), picks their next steps (Aarseth 1985 criterion, cited in
 * Sect. 3.1-3.2) and sends them back with g6_set_j_particle. */

typedef struct g6h_sim g6h_sim;

/* Create a simulation of n particles (masses m[n], positions x[n][3],
 * velocities v[n][3], copied) on cluster id `clusterid` (opened by the
 * caller).  eta: accuracy parameter; eta_s: initial-step parameter (<= 0:
 * eta / 10); dt_max: largest step (a power of two); dt_min: smallest.
 * Computes the initial force with one full sweep.  Returns NULL on error
 * (*err receives the code when err != NULL). */
g6h_sim *g6h_create(int clusterid, int n, const double *m, const double *x,
                    const double *v, double eps2, double eta, double eta_s,
                    double dt_max, double dt_min, int *err);

/* Advance block steps until every particle reaches t_end (a multiple of
 * dt_max).  Returns 0 or a negative error. */
int g6h_run(g6h_sim *s, double t_end);

/* As g6h_run, but stop after at most max_blocks block steps.  Returns the
 * number of block steps taken (fewer than max_blocks once every particle
 * has reached t_end) or a negative error.  Between calls the particles sit
 * at their own last block times (g6h_get_state: t, dt), as in GRAPE-style
 * codes between blocks. */
long long g6h_run_blocks(g6h_sim *s, double t_end, long long max_blocks);

/* The driver's corrector and time-step choice for n particles that reach
 * the block time t_blk together (Sect. 2; Makino & Aarseth 1992 corrector,
 * Aarseth 1985 criterion with a'' taken at the end of the step, power-of-two
 * quantisation that may double only at commensurate times).  Per particle:
 * t0, dt = time and step of its last correction; xp, vp [n][3] = predicted
 * state at t_blk, overwritten with the corrected x1, v1; (a0, j0) force at
 * t0 and (a1, j1) at t_blk [n][3]; dt_new = next step, -1 where it would fall
 * below dt_min.  Returns the number of such particles, or G6_EINVAL. */
int g6h_correct_block(int n, double t_blk, const double *t0, const double *dt,
                      double eta, double dt_max, double dt_min, double *xp,
                      double *vp, const double *a0, const double *j0,
                      const double *a1, const double *j1, double *dt_new);

/* g6h_correct_block with a time-step choice that allows for a relative
 * force error force_noise (>= 0; 0 gives g6h_correct_block): before
 * Aarseth's criterion, the magnitudes of the second and third derivatives
 * are reduced by what force errors of that relative size alone can put into
 * them through the corrector's differences (up to (24 na + 12 h nj)/h^3 and
 * (36 na + 18 h nj)/h^2 with na = force_noise |a|, nj = force_noise |j|), so
 * that force noise is not read as structure that shrinks the steps (Sect.
 * 3.1: with low-precision forces small steps tend to become much smaller).
 * The request is the larger of the plain one and the reduced one, so the
 * allowance never shortens a step.  Not in the paper; off unless asked for. */
int g6h_correct_block_ex(int n, double t_blk, const double *t0, const double *dt,
                         double eta, double dt_max, double dt_min, double *xp,
                         double *vp, const double *a0, const double *j0,
                         const double *a1, const double *j1, double *dt_new,
                         double force_noise);

/* Use g6h_correct_block_ex's time-step choice with relative force error
 * rel (0 <= rel < 1; 0, the default, is the plain criterion).  Returns 0 or
 * G6_EINVAL. */
int g6h_set_force_noise(g6h_sim *s, double rel);

/* Copy the current state out (any pointer may be NULL): x, v, acc, jerk
 * [n][3]; t, dt [n]. */
int g6h_get_state(const g6h_sim *s, double *x, double *v, double *acc,
                  double *jerk, double *t, double *dt);

/* Kinetic + potential energy of the synchronised system, the potential
 * from one full force sweep through the library.  Returns 0 or an error. */
int g6h_energy(g6h_sim *s, double *e_kin, double *e_pot);

/* Counters: block steps, sum of block sizes, and a 64-bin histogram of
 * floor(log2(block size)) (hist may be NULL). */
int g6h_stats(const g6h_sim *s, long long *nblocks, long long *nactive,
              long long *hist);

/* Wall-clock seconds g6h_run spent choosing blocks (scheduler, host
 * prediction), in the force calls (firsthalf + lasthalf) and in correcting
 * and sending back the corrected particles.  Any pointer may be NULL. */
int g6h_profile(const g6h_sim *s, double *sec_sched, double *sec_force,
                double *sec_correct);

/* Neighbour lists in the driver (Sect. 4): with h2 > 0 every block step's
 * force call also builds the active particles' lists of neighbours within
 * unsoftened |r|^2 < h2 and reads them back (g6_read_neighbour_list /
 * g6_get_neighbour_list); h2 = 0 turns them off (the default).  The energy
 * sweep never builds lists.  Returns 0, G6_EINVAL or G6_ENOMEM. */
int g6h_set_neighbour_radius(g6h_sim *s, double h2);

/* Lists read back so far, their total length (entries kept, at most the
 * context's list length per list) and how many overflowed it.  Any pointer
 * may be NULL. */
int g6h_neighbour_stats(const g6h_sim *s, long long *lists, long long *entries,
                        long long *overflowed);

void g6h_destroy(g6h_sim *s);

/* Checkpoint: write the driver's whole state (particles, block scheduler in
 * its order, counters and parameters) to `path` (written to path.tmp, then
 * renamed over path).  Returns 0, G6_EINVAL or G6_EIO. */
int g6h_checkpoint(const g6h_sim *s, const char *path);

/* Resume: rebuild a driver from a checkpoint on cluster id `clusterid`
 * (opened by the caller, any precision) and send every particle's state to
 * its j-memory; no force is computed.  Continuing a restored driver with the
 * same library settings reproduces the original run.  Returns NULL on error
 * (*err: G6_EIO if the file cannot be read, G6_EINVAL if its content is not
 * a consistent checkpoint (magic, sizes, parameters, scheduler times,
 * every particle filed once, hash), G6_ENOMEM, or the error of the first
 * failing library call). */
g6h_sim *g6h_restore(int clusterid, const char *path, int *err);

/* ------------------------------------------------ batches of clusters ----
 * Many independent star clusters in one device (Sect. 2: one library
 * instance per cluster id, each with its own j-memory and block time).  A
 * batch keeps the j-memory of ncl clusters side by side; one batch
 * calculation computes, for every cluster k, the forces on its ni[k]
 * i-particles at its own block time t_blk[k] with its own softening
 * eps2[k] (Eq. 1 - Eq. 3, DS arithmetic), all clusters in one launch
 * sequence: the j-update fused into the prediction, one force kernel whose
 * work line concatenates every cluster's (i-tile, j-tile) pairs, and the
 * partial-sum reduction.  Cluster k's particle q lives at j-address q
 * (0 <= q < nj[k]); particle indices, self-exclusion and nearest neighbours
 * are per cluster.  Neighbour lists are not available on batches.
 * Threading: g6x_batch_set_j / _set_j_many calls for different clusters may
 * run concurrently; every other call on a batch takes it alone. */

typedef struct g6x_batch g6x_batch;

/* Create a batch of ncl clusters with nj[k] >= 1 j-particles each.
 * precision: G6X_PREC_DS or G6X_PREC_DS_X64.  variant: batch force kernel
 * (0 .. 7: 16x16x1, 16x16x2, 32x8x2, 64x4x2, 128x1x2, 8x32x1, 8x32x2,
 * 4x64x2 threads along i x threads along j x i-particles per thread; the
 * i-tile is the product of the first and last) for a one-class schedule, or -1 for the default
 * two-class schedule (kernel 0 for active sets of up to 32, kernel 3
 * above).  grid_mul: CTAs = SMs x resident CTAs per SM x grid_mul (0 = 1
 * for a given variant, 2 for the wide kernel of the default schedule;
 * at most 16).  Device memory comes from
 * the allocator set with g6x_set_allocator; i-records, results and the
 * per-step tables are in mapped pinned host memory.  Returns NULL on error
 * (*err = G6_EINVAL, G6_ENOMEM, G6_ENODEV or G6_EIO). */
g6x_batch *g6x_batch_create(int ncl, const int nj[], int precision, int variant,
                            int grid_mul, int *err);
int g6x_batch_destroy(g6x_batch *b);

/* Schedule: clusters whose active set has at most `threshold` particles
 * are computed by force kernel small_variant, the others by large_variant
 * (both as for g6x_batch_create), each over its own work line with its own
 * grid multiplier (1 .. 16); the two kernels run concurrently.
 * large_variant = -1: one class, small_variant for every cluster (threshold
 * ignored).  Waits for the batch's work, reallocates the partial-sum
 * buffers and re-captures the graph at the next call.  Returns 0,
 * G6_EINVAL or G6_ENOMEM. */
int g6x_batch_set_schedule(g6x_batch *b, int small_variant, int small_grid_mul,
                           int threshold, int large_variant, int large_grid_mul);

/* Current schedule: {small_variant, small_grid_mul, threshold,
 * large_variant, large_grid_mul} (threshold 0 and large_variant -1 for a
 * one-class schedule). */
int g6x_batch_get_schedule(const g6x_batch *b, int sched[5]);

/* Schedule autotuner: times every one-class schedule (each kernel, grid
 * multiplier 1 and 2) and the two-class schedules (narrow kernel x wide
 * kernel x thresholds 8 .. 128) on npat active-set patterns ni[npat][ncl]
 * (graph mode, reps passes, at block times t_blk[ncl] with softenings
 * eps2[ncl]) and keeps the fastest.  The calls compute on the batch's
 * current j-memory and i-records and overwrite its results; staged records
 * are applied by the first call.  sched (may be NULL) receives the chosen
 * schedule as g6x_batch_get_schedule, best_ms (may be NULL) its mean
 * milliseconds per call.  Returns 0 or an error. */
int g6x_batch_autotune(g6x_batch *b, int npat, const int ni[], const double eps2[],
                       const double t_blk[], int reps, int sched[5], double *best_ms);

/* Host pointer to cluster cl's i-record array (nj[cl] records, mapped
 * memory written by the caller before g6x_batch_calc; index = the
 * particle's index within the cluster, used for self-exclusion; h2 unused),
 * and to its result array (g6x_out, valid after g6x_batch_calc returns;
 * nnb is the nearest neighbour's index within the cluster).  NULL on a bad
 * batch or cluster. */
g6x_irec *g6x_batch_irecs(g6x_batch *b, int cl);
const g6x_out *g6x_batch_results(const g6x_batch *b, int cl);

/* Stage particle `address` of cluster cl (same arguments and meaning as
 * g6_set_j_particle; index is the particle's index within the cluster).
 * The record reaches j-memory at the next g6x_batch_calc.  Returns 0,
 * G6_EINVAL or G6_ENOMEM. */
int g6x_batch_set_j(g6x_batch *b, int cl, int address, int index, double tj,
                    double mass, const double j6[3], const double a2[3],
                    const double v[3], const double x[3]);

/* Stage n particles of cluster cl at once: address[n], index[n], tj[n],
 * mass[n], j6, a2, v, x [n][3] (same meaning as g6x_batch_set_j).  Checks
 * every address and index before staging any.  Returns 0, G6_EINVAL or
 * G6_ENOMEM. */
int g6x_batch_set_j_many(g6x_batch *b, int cl, int n, const int address[],
                         const int index[], const double tj[], const double mass[],
                         const double j6[], const double a2[], const double v[],
                         const double x[]);

/* One batch calculation: per cluster k, predict its j-particles to t_blk[k]
 * (Eq. 1, Eq. 2) and compute forces on its first ni[k] i-records
 * (0 <= ni[k] <= nj[k]; 0 = idle this step) with softening eps2[k].
 * mode 0: one CUDA-graph replay of the three kernels (captured at the first
 * call); 1: the same three kernels as plain launches; 2: one launch
 * sequence per active cluster.  Blocks until the results are in.  Returns 0,
 * G6_EINVAL, G6_ETIMEDOUT or G6_EIO. */
int g6x_batch_calc(g6x_batch *b, const double t_blk[], const double eps2[],
                   const int ni[], int mode);

/* CUDA-event timing of every batch calculation (enable = 1 resets the
 * totals): the GPU time of the launch sequence, from before the table copy
 * to after the last kernel, summed over calls. */
int g6x_batch_set_timing(g6x_batch *b, int enable);
int g6x_batch_get_timing(const g6x_batch *b, double *gpu_ms, long long *calls);

/* Kernels and copies launched by the batch: a graph replay counts one table
 * copy and three (one class) or five (two classes) kernels as 1 + 2 x
 * classes; a per-cluster sequence counts three per active cluster. */
long long g6x_batch_launch_count(const g6x_batch *b);

/* Hermite driver over a batch: every cluster runs the block-time-step
 * integration of g6h_run with its own block scheduler; one g6hb_step
 * advances each cluster that has not reached t_end by one of its block
 * steps, all clusters' forces in one g6x_batch_calc. */
typedef struct g6hb_sim g6hb_sim;

/* ncl clusters of n[k] particles; m, x, v hold the clusters one after
 * another (m[sum n], x and v [sum n][3]); eps2[k] per cluster; eta, eta_s,
 * dt_max, dt_min as for g6h_create; variant and grid_mul as for
 * g6x_batch_create; mode as for g6x_batch_calc.  Computes the initial
 * forces.  NULL on error. */
g6hb_sim *g6hb_create(int ncl, const int n[], const double *m, const double *x,
                      const double *v, const double eps2[], double eta,
                      double eta_s, double dt_max, double dt_min, int variant,
                      int grid_mul, int mode, int *err);

/* One batch step up to t_end: returns the number of clusters that stepped
 * (0 once every cluster has reached t_end) or a negative error. */
int g6hb_step(g6hb_sim *s, double t_end);

/* Steps until every cluster reaches t_end (a multiple of dt_max). */
int g6hb_run(g6hb_sim *s, double t_end);

/* The driver's batch (for g6x_batch_set_timing and the like); NULL for a
 * NULL driver. */
g6x_batch *g6hb_batch(g6hb_sim *s);

/* As g6h_set_force_noise, for every cluster of a batch driver. */
int g6hb_set_force_noise(g6hb_sim *s, double rel);

/* Change the launch mode (0, 1, 2 as for g6x_batch_calc). */
int g6hb_set_mode(g6hb_sim *s, int mode);

/* Tune the batch schedule (g6x_batch_autotune) on the active-set patterns
 * of the driver's last (up to 64) batch steps.  Returns G6_EBUSY before the
 * first step. */
int g6hb_autotune(g6hb_sim *s, int reps, int sched[5], double *best_ms);

/* Set the batch schedule (as g6x_batch_set_schedule). */
int g6hb_set_schedule(g6hb_sim *s, int small_variant, int small_grid_mul,
                      int threshold, int large_variant, int large_grid_mul);

/* Counters: batch steps, sum of active particles, sum over steps and
 * clusters of ni x nj, seconds in g6x_batch_calc and on the host. */
int g6hb_stats(const g6hb_sim *s, long long *nsteps, long long *nactive,
               long long *interactions, double *sec_gpu, double *sec_host);

/* State of every particle in creation order: x, v [sum n][3], t [sum n]. */
int g6hb_get_state(const g6hb_sim *s, double *x, double *v, double *t);
/* The same with the acceleration and jerk [sum n][3] of each particle's
 * last correction and its time step dt [sum n] (any pointer may be NULL):
 * between batch steps a particle sits at its own last block time t and its
 * next one is t + dt (Sect. 2.1). */
int g6hb_get_state_ex(const g6hb_sim *s, double *x, double *v, double *acc, double *jerk,
                      double *t, double *dt);

void g6hb_destroy(g6hb_sim *s);

#ifdef __cplusplus
}
#endif
#endif /* G6GB_H */
