/*
 * sp.h -- C ABI of the region-scheduled ("semi-parallel") evolution of a
 * complex scalar string field on one GB300.
 *
 * The method (Blanco-Pillado, Olum, Shlaer, "A new parallel simulation
 * technique", Sec. 1-4): spacetime is cut by null surfaces into many small
 * regions that receive data only through initial surfaces and emit it only
 * through final surfaces, so each region can be evolved on its own as soon as
 * its predecessors are done, and a manager hands ready regions to workers
 * (Sec. 4).  Here a region is a pyramid, inverted pyramid or wedge of B^3
 * lattice cells and B/2 leapfrog steps; the manager is a device work queue
 * and the workers are the CTAs of one persistent kernel.  The model equation,
 * in conformal time tau with a = (tau / tau_ref)^nu, is
 *
 *   phi'' + 2 (nu / tau) phi' - Lap7 phi + a^2 lambda (|phi|^2 - eta^2) phi = 0,
 *
 * advanced by the staggered leapfrog (FP32 with a Kahan-compensated drift).
 *
 * Conventions for every entry point:
 *   - Return value: SP_OK (0) or a negative SP_E* code; sp_strerror() names
 *     it.  No C++ exception crosses this boundary.
 *   - Device pointers are plain CUDA device addresses of the current device.
 *     Host pointers are ordinary (preferably pinned) host memory.
 *   - Work is enqueued on the stream given at creation.  Asynchronous device
 *     errors (a bounded wait that gave up, a CUDA fault) are reported by the
 *     next call that synchronises (sp_evolve without SP_ASYNC,
 *     sp_read_surface).
 *   - State of one simulation, both arrays with site index
 *     x + n[0] * (y + n[1] * z) (x fastest):
 *       phi : float2[sites]  (Re phi, Im phi) at level n;
 *       pic : float4[sites]  (Re pi, Im pi, Re c, Im c): pi = phi' at level
 *             n - 1/2 and c, the Kahan carry of phi at level n.
 *     24 bytes per site in all.
 */
#ifndef SP_H
#define SP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- error codes ---- */
#define SP_OK 0
#define SP_EINVAL (-1)          /* bad argument or call order */
#define SP_ENOMEM (-2)          /* device or host allocation failed */
#define SP_ECUDA (-3)           /* a CUDA runtime call failed */
#define SP_EUNSTABLE (-4)       /* leapfrog stability bound violated by the plan */
#define SP_ETIMEOUT (-5)        /* a bounded device wait gave up */
#define SP_ENONFINITE (-6)      /* non-finite field detected by a diagnostic */
#define SP_EFAULT_INJECTED (-7) /* a host-injected region failure was recorded */
#define SP_ENOTPLANNED (-8)     /* sp_evolve before sp_region_plan */
#define SP_ESCRATCH (-9)        /* sp_sweep_noalloc: grid or step count beyond its fixed scratch */

/* ---- flags of sp_evolve ---- */
#define SP_ASYNC 1u      /* return without synchronising the stream */
#define SP_MONOLITHIC 2u /* whole-grid sweep, one launch per step (comparator) */
#define SP_RESTART 4u    /* treat the current state as level 0 (tau = tau0) */
#define SP_TRACE 8u      /* record (start, end) globaltimer ns of every region (SP_SURF_TRACE) */
#define SP_TIMING 16u    /* record CUDA events around each launch of the call (SP_SURF_TIMING) */
#define SP_FEATURES 32u  /* compute the cost-model features of every region of the call (SP_SURF_FEATURES) */

/* ---- what of sp_read_surface / sp_write_surface ---- */
#define SP_SURF_STATE 0   /* phi (sites float2) then pic (sites float4): 24 * sites bytes */
#define SP_SURF_DIAG 1    /* one sp_diag */
#define SP_SURF_TRACE 2   /* per-region (start, end) ns of the last region launch */
#define SP_SURF_WINDING 3 /* int8 plaquette windings [3][sites] */
#define SP_SURF_PLAN 4    /* one sp_plan_info */
#define SP_SURF_TIMING 5  /* double[3]: ms of the queue reset, the region kernel and the
                             remainder sweep of the last SP_TIMING call (events on the stream) */
#define SP_SURF_LEVEL 7    /* int64 (host memory): the simulation's current level n; readable and
                              writable -- a checkpoint is SP_SURF_STATE plus SP_SURF_LEVEL */
#define SP_SURF_FEATURES 6 /* float[regions][SP_MODEL_FEATURES]: cost-model inputs of the sim's regions
                              in the last SP_FEATURES (or learned-order) call, in region-id order
                              (the order of SP_SURF_TRACE) */

/* ---- sp_region_plan: base_B / block_shape chosen by measurement ---- */
#define SP_AUTOTUNE (-1)

/* ---- sp_params.precision ---- */
#define SP_FP32_KAHAN 0 /* FP32 state (phi, pi, Kahan carry of phi), FP32 site update with explicit fused
                           multiply-adds, per-level coefficients computed in FP64 and rounded once */

/* ---- region ordering of sp_region_plan ---- */
#define SP_ORDER_STATIC 0  /* release order of the dependency DAG */
#define SP_ORDER_LEARNED 1 /* cost-model priority (results are identical) */

/* ---- sp_set_option ---- */
#define SP_OPT_WAIT_LIMIT_NS 1      /* bound of every device-side wait, ns (default 2e9; 1e6 .. 6e10) */
#define SP_OPT_FAULT_DROP_RELEASE 2 /* inject a failure: the region with this id in the next region
                                       launches (ids as in SP_SURF_TRACE, simulations concatenated)
                                       finishes but never releases its successors, so the launch ends
                                       with SP_ETIMEOUT after the wait limit; -1 clears */
#define SP_OPT_GRAPHS 3             /* 1 (default): capture region calls into CUDA graphs on
                                       non-legacy streams; 0: launch directly */
#define SP_OPT_REGION_SHAPE 5       /* region geometry, applied by the next sp_region_plan:
                                       SP_SHAPE_SPLIT (default) or SP_SHAPE_LATTICE */
#define SP_OPT_MAILBOX_SLOTS 4      /* sloped-surface mailboxes, applied by the next sp_region_plan:
                                       1 (default): one slot for every band, with each region also
                                       waiting for the previous band's readers of the mailboxes it
                                       writes; 2: a ring of two band slots, twice the memory
                                       (sp_plan_info.mailbox_bytes).  Results are identical. */

/* ---- region geometry (SP_OPT_REGION_SHAPE) ----
 * SP_SHAPE_SPLIT: products of 1-D diamonds (pyramids, inverted pyramids and
 *   wedges of B^3 cells, B/2 steps per band), surfaces routed through
 *   mailboxes.
 * SP_SHAPE_LATTICE: the paper's own lattice of 4-cubes with time along the
 *   main diagonal (Sec. 2, Figs. 2-5): one congruent region type of
 *   16 s^4 site-updates over 4s levels with four initial and four final
 *   faces, B = 4s the cube's edge; four predecessors and four successors per
 *   region (Fig. 2's layers).  Regions read and write the state arrays in
 *   place (phi at odd levels of a call in a second array of 8 bytes per
 *   site), so no mailbox is allocated; any step count runs as regions.
 *   Results are bit-identical to the split tiling and the sweep. */
#define SP_SHAPE_SPLIT 0
#define SP_SHAPE_LATTICE 1

/* ---- region cost model ---- */
#define SP_MODEL_FEATURES 16
#define SP_MODEL_PARAMS 5313 /* W1[64][16] b1[64] W2[64][64] b2[64] W3[64] b3[1], FP32 */
typedef struct sp_model sp_model; /* opaque */

typedef struct sp_grid sp_grid; /* opaque */

/* Physical and numerical parameters of one simulation. */
typedef struct {
    int32_t n[3];        /* grid sides (sites); each a multiple of the region base B, n/B >= 2 */
    double dx;           /* lattice spacing (> 0) */
    double dt;           /* conformal time step (> 0) */
    double lambda;       /* quartic coupling (>= 0) */
    double eta;          /* vacuum expectation value (>= 0) */
    double nu;           /* expansion exponent: a = (tau / tau_ref)^nu; 0 flat, 1 radiation, 2 matter */
    double tau0;         /* conformal time at level 0 (> 0) */
    double tau_ref;      /* time at which a = 1 (> 0); normally tau0 + steps * dt */
    int32_t damp_steps;  /* initial levels with the velocity discarded each step (tau frozen at tau0) */
    int32_t precision;   /* arithmetic of the evolution: SP_FP32_KAHAN (0), the only one built */
} sp_params;

/* Diagnostics of one simulation at its current level. */
typedef struct {
    int64_t level;          /* current level n */
    double tau, a;          /* conformal time and scale factor at that level */
    double kinetic;         /* sum |pi|^2 (pi at n - 1/2) */
    double gradient;        /* sum over forward links |phi(x+e) - phi(x)|^2 / dx^2 */
    double potential;       /* sum a^2 (lambda / 2) (|phi|^2 - eta^2)^2 */
    double total;           /* kinetic + gradient + potential */
    int64_t pierced[3];     /* plaquettes with nonzero winding, by normal axis x, y, z */
    int64_t abs_winding;    /* sum |W| over all plaquettes */
    int64_t net_winding[3]; /* sum W by normal axis (0 on a periodic grid) */
    double string_length;   /* (pierced[0] + pierced[1] + pierced[2]) * dx */
} sp_diag;

/* Plan summary of one simulation (traffic is of this design, per band;
 * threads, ctas_per_sm and grid are those of the launch of its base). */
typedef struct {
    int32_t base_B, threads, ctas_per_sm, grid;
    int64_t regions_per_band;
    int64_t updates_per_band;
    int64_t bytes_read_per_band;
    int64_t bytes_written_per_band;
    double bytes_per_update;
    int64_t mailbox_bytes;
    int32_t autotuned;       /* 1 if base_B or block_shape was SP_AUTOTUNE */
    int32_t tune_candidates; /* candidates the autotuner timed */
    double tune_best_ms;     /* its trial time of the chosen candidate (16 steps) */
    double tune_default_ms;  /* its trial time of the default choice, 0 if not timed */
    int32_t mailbox_slots;   /* 2: ring of two band slots; 1: one slot for every band (0: lattice) */
    int32_t region_shape;    /* SP_SHAPE_SPLIT or SP_SHAPE_LATTICE; for a lattice plan "band" reads
                                "layer" (s levels: 4 M_x M_y M_z regions, N_d = B M_d) and
                                mailbox_bytes holds the odd-level phi array */
} sp_plan_info;

/*
 * sp_grid_create -- describe n_sims independent simulations.
 * Paper Sec. 2.1: a region is evolved from data on its initial surfaces
 * alone, and the first regions read the initial time slice itself; the
 * state given here is that slice (level 0) for every simulation.
 *   p         : array of n_sims parameter sets (host memory, copied).
 *   state_dev : NULL, or 2 * n_sims device pointers (phi, pic of sim 0, then
 *               sim 1, ...): phi float2[sites] (8-byte aligned), pic
 *               float4[sites] (16-byte aligned).  The caller keeps ownership
 *               and must keep them alive until sp_destroy.  With NULL the
 *               library allocates zeroed state it frees itself.  Between
 *               calls the state holds (phi_n, pi_{n-1/2}, c_n).
 *   cuda_stream : cudaStream_t used for all work (NULL = legacy stream).
 *   out       : receives the handle.
 * Errors: SP_EINVAL (bad parameters), SP_ENOMEM, SP_ECUDA.
 */
int sp_grid_create(const sp_params *p, int32_t n_sims, void *const *state_dev, void *cuda_stream, sp_grid **out);

/*
 * sp_region_plan -- build the region tiling, the dependency DAG and the
 * surface routing tables (paper Sec. 2 geometry and Sec. 3 sizing), and size
 * the persistent launch.
 *   base_B     : region base in cells (4, 8, 16 or 32; B/2 steps per band);
 *                0 to take 16 where it divides every side of a simulation,
 *                else 8; SP_AUTOTUNE to time the policies (all 8, 16 where
 *                possible, 32 where possible) and keep the fastest.  Every
 *                n[d] must be a multiple of B with n[d] / B >= 2.
 *                With SP_SHAPE_LATTICE: the 4-cube edge B = 4s, s = 1..6
 *                (4, 8, 12, 16, 20 or 24; 4s levels per region); every n[d]
 *                a multiple of B; 0 takes 16 where it divides, else 8, else
 *                4; SP_AUTOTUNE times the sizes that divide every side.
 *   block_shape: worker threads per CTA (64, 128, 256, 320, 384, 480, 512 or 768;
 *                lattice plans: 64, 128, 192, 256 or 512, one region per CTA
 *                and no manager warp (default: 128 up to s = 4, 256 at
 *                s = 5, 512 at s = 6);
 *                every worker taking every step of a region); one manager
 *                warp is added.  0 for the default of each base (64 for
 *                bases 4 and 8, 384 for 16); SP_AUTOTUNE to time the
 *                candidates for the largest base (64, 128 for base 8; 320,
 *                384, 480 for base 16), smaller bases keeping their default.
 *                A value applies to every base.
 *                The autotuner runs 16-step calls on scratch copies of the
 *                current state (sides above 128 cells are cut to 128 or 120),
 *                on the grid's stream; the state itself is not modified.
 *   order      : SP_ORDER_STATIC (ready regions are popped in the order they
 *                became ready) or SP_ORDER_LEARNED (each call predicts every
 *                region's cost from its features with the model at
 *                model_path and pops the predicted-expensive quarter first,
 *                then the next quarter, ...).  The order never changes results.
 *   model_path : file written by sp_model_save; required for SP_ORDER_LEARNED.
 * Errors: SP_EINVAL, SP_ENOMEM, SP_ECUDA.
 */
int sp_region_plan(sp_grid *g, int32_t base_B, int32_t block_shape, int32_t order, const char *model_path);

/*
 * sp_evolve -- advance every simulation by n_steps leapfrog steps.
 * Paper Sec. 4: a manager holds the pool of regions whose predecessors are
 * done and hands one to each worker that reports its previous region
 * finished; here the pool is a device work queue and the workers are the
 * CTAs of one persistent launch per region base.
 * Whole bands of B/2 steps run as regions in one persistent launch per
 * distinct base (largest base first, each launch sized for its base); a
 * remainder of fewer than B/2 steps runs as whole-grid steps with the same
 * arithmetic.  SP_MONOLITHIC runs every step as a whole-grid sweep (bit-exact
 * with the region path).  Unless SP_ASYNC is given the call synchronises the
 * stream and reports device errors.
 * Errors: SP_EINVAL, SP_ENOTPLANNED, SP_EUNSTABLE (dt^2 (12/dx^2 + 2 lambda
 * eta^2 a^2) >= 4 at some level), SP_ETIMEOUT, SP_ECUDA.
 */
int sp_evolve(sp_grid *g, int64_t n_steps, uint32_t flags);

/*
 * sp_set_option -- set one of the SP_OPT_* options above.
 * Errors: SP_EINVAL.
 */
int sp_set_option(sp_grid *g, int32_t option, int64_t value);

/*
 * sp_read_surface -- copy out one simulation's state or diagnostics.
 * Paper Sec. 2.2: the final surfaces that regions write are what later
 * regions (and the user) read; after a call the inverted pyramids' tops form
 * the whole field at the current level, which is what SP_SURF_STATE returns.
 * The string diagnostics follow the paper's Sec. 5 output (string length).
 *   what : SP_SURF_STATE, SP_SURF_DIAG, SP_SURF_TRACE, SP_SURF_WINDING or
 *          SP_SURF_PLAN; dst_bytes must be at least the size of that item.
 *   dst_is_device : nonzero if dst is device memory.
 * Synchronises the stream.  Errors: SP_EINVAL, SP_ETIMEOUT (pending device
 * error), SP_ECUDA.
 */
int sp_read_surface(const sp_grid *g, int32_t sim, int32_t what, void *dst, size_t dst_bytes, int32_t dst_is_device);

/*
 * sp_write_surface -- load one simulation's state (what = SP_SURF_STATE:
 * paper Sec. 2.1's initial slice, or a checkpoint: Sec. 7 notes that
 * surfaces are natural restart points)
 * phi then pic, 24 * sites bytes) from host or device memory, enqueued on the
 * grid's stream; or set its current level (what = SP_SURF_LEVEL, one int64 in
 * host memory), which selects tau, a and the friction of the next steps.
 * Restoring SP_SURF_STATE and SP_SURF_LEVEL from a checkpoint resumes a run
 * bit-exactly.  Errors: SP_EINVAL, SP_ECUDA.
 */
int sp_write_surface(sp_grid *g, int32_t sim, int32_t what, const void *src, size_t src_bytes, int32_t src_is_device);

/*
 * Region cost model (paper Sec. 4: the manager issues regions so that the
 * expensive ones do not finish last).  A 16-64-64-1 ReLU network in FP32
 * predicting log(region time in microseconds) from the 16 features that
 * SP_FEATURES records (SP_SURF_FEATURES); trained on the GPU by minibatch
 * Adam (beta 0.9 / 0.999, eps 1e-8) on the mean squared error.
 *
 * sp_model_create  -- He-uniform weights from seed (weight k: SplitMix64
 *                     output k of the stream at seed, (2u-1) sqrt(6/fan_in)),
 *                     zero biases; work goes to cuda_stream.
 * sp_model_get_params / sp_model_set_params -- SP_MODEL_PARAMS floats (host),
 *                     and optionally the 3 bucket thresholds (non-increasing).
 *                     Setting parameters resets the Adam state.
 * sp_model_predict -- y_dev[i] = network(x_dev[16 i .. 16 i + 15]) (device).
 * sp_model_grad    -- gradient (host, SP_MODEL_PARAMS floats) and loss of the
 *                     mean squared error over n samples (device x, y).
 * sp_model_adam_step -- one Adam step with the given gradient (host).
 * sp_model_train   -- epochs x ceil(n / batch) Adam steps on minibatches in
 *                     the order order_host (epochs * n sample indices), or,
 *                     when it is NULL, per epoch e the stable argsort of
 *                     uniforms 2^42 + e 2^32 + i of the stream order_seed.
 *                     losses_host (optional) receives each minibatch's loss
 *                     before its step.  Afterwards the bucket thresholds are
 *                     set to the 75th, 50th and 25th percentiles of the
 *                     network's predictions on the training set.
 * sp_model_save / sp_model_load -- parameters and thresholds in a file.
 * All synchronise the model's stream.  Errors: SP_EINVAL, SP_ENOMEM, SP_ECUDA.
 */
int sp_model_create(uint64_t seed, void *cuda_stream, sp_model **out);
int sp_model_destroy(sp_model *m);
int sp_model_get_params(sp_model *m, float *params_host, float *thresholds_host);
int sp_model_set_params(sp_model *m, const float *params_host, const float *thresholds_host);
int sp_model_predict(sp_model *m, const float *x_dev, int64_t n, float *y_dev);
int sp_model_grad(sp_model *m, const float *x_dev, const float *y_dev, int64_t n, float *grad_host, double *loss);
int sp_model_adam_step(sp_model *m, const float *grad_host, float lr, float beta1, float beta2, float eps);
int sp_model_train(sp_model *m, const float *x_dev, const float *y_dev, int64_t n, int32_t epochs, int32_t batch,
                   float lr, uint64_t order_seed, const int32_t *order_host, float *losses_host);
int sp_model_save(sp_model *m, const char *path);
int sp_model_load(const char *path, void *cuda_stream, sp_model **out);

/*
 * sp_sweep_noalloc -- advance one simulation by n_steps whole-grid leapfrog
 * steps without allocating any memory.  (The paper has no counterpart: this
 * entry point serves callers that may not allocate device memory -- programs
 * that own all device memory through their own fixed pools, plug-ins that
 * must not grow the process's footprint, latency-critical paths.)
 *   p         : parameters of the simulation (host memory).
 *   phi_dev, pic_dev : its state in the layout above, updated in place.
 *   level0    : level of the state on entry (selects tau, a and friction).
 *   n_steps   : steps to take; the work is enqueued on cuda_stream and the
 *               call returns without synchronising.
 * Results are bit-identical to sp_evolve(..., SP_MONOLITHIC) from the same
 * state and level.  Scratch: a phi ping-pong buffer of at most
 * SP_NOALLOC_MAX_SITES sites (2 MiB) and SP_NOALLOC_MAX_STEPS per-level
 * coefficients (128 KiB), in fixed device arrays that every GPU loading the
 * library holds until exit.  The first call on a device looks up those
 * arrays' device addresses (once per device); make it before any stream
 * capture.  With CUDA's lazy module loading the arrays are created on a
 * device when this first call loads the library's device code there, so make
 * that first call early, before the caller's own pools take the device's
 * memory.  All calls share the arrays: calls whose work overlaps on the GPU
 * (other streams, other threads) race and must be serialised by the caller.
 * Calls no cudaMalloc, cudaFree or allocating library routine, and uses no
 * host heap: the coefficients travel as kernel arguments.
 * Errors: SP_EINVAL (also for a side outside [4, 16384]), SP_ESCRATCH (more than SP_NOALLOC_MAX_SITES sites or
 * SP_NOALLOC_MAX_STEPS steps), SP_EUNSTABLE, SP_ECUDA.
 */
#define SP_NOALLOC_MAX_SITES 262144
#define SP_NOALLOC_MAX_STEPS 8192
int sp_sweep_noalloc(const sp_params *p, void *phi_dev, void *pic_dev, int64_t level0, int64_t n_steps,
                     void *cuda_stream);

/*
 * sp_lattice_call_bytes -- what a call of n_steps levels moves with lattice
 * regions of edge B = 4s (SP_SHAPE_LATTICE): site-updates and HBM bytes read
 * and written by one region column (one region position in every layer of
 * the call; a layer holds 4 M_x M_y M_z regions), including the whole-state
 * loads of the regions cut by the call's first level and the whole-state
 * exports of those cut by its last.  bytes / updates is the call's
 * algorithmic bytes per site-update (paper Sec. 3: surface over volume).
 * Host only, no device work.  Errors: SP_EINVAL (B not 4..24 in steps of 4,
 * n_steps < 1, a NULL output).
 */
int sp_lattice_call_bytes(int32_t B, int64_t n_steps, int64_t *updates, int64_t *bytes_read, int64_t *bytes_written);

/*
 * sp_measure_peaks -- measured on-chip peaks of the current device, for the
 * roofline lines of the region kernel (its shared-memory traffic and its
 * FP32 arithmetic; the HBM line uses a measured copy bandwidth): the
 * shared-memory read bandwidth of the whole device (GB/s: every SM reading
 * 16-byte words without bank conflicts) and the FP32 fused multiply-add
 * throughput (TFLOP/s, 2 flops per FMA).  Each is one timed launch after a
 * warm-up on cuda_stream; the call synchronises.  The paper has no
 * counterpart (its cost figures are CPU times, Sec. 6).
 * Errors: SP_EINVAL (NULL output), SP_ENOMEM, SP_ECUDA.
 */
int sp_measure_peaks(void *cuda_stream, double *smem_gbs, double *fp32_tflops);

/* sp_destroy -- free everything the library allocated (not caller state):
 * plan, mailboxes, work queue, scratch.  Paper Sec. 4: when the pool of
 * regions is empty the manager retires its workers; this is the host-side end
 * of that life cycle.  Synchronises the grid's stream first.
 * Errors: SP_EINVAL (NULL handle). */
int sp_destroy(sp_grid *g);

/* sp_strerror -- static description of an error code. */
const char *sp_strerror(int code);

#ifdef __cplusplus
}
#endif

#endif /* SP_H */
