/*
 * me.h -- C ABI of the GB300 event-parallel NLO matrix-element library.
 *
 * The library evaluates, for a batch of independent phase-space points, the
 * tree-level quantities that dominate fixed-order NLO run time (arXiv:2503.07439,
 * Sec. 4.1 and Fig. 1: Born, real-emission and counterterm amplitudes; Sec. 4.2:
 * all of them are tree-level amplitudes) behind the multi-event interface of
 * Sec. 4.4 (step 1 of the work plan), with the branch-free per-point flow of
 * Sec. 4.3, Algorithm 2.
 *
 * Conventions for every entry point:
 *  - momenta: float64 structure-of-arrays, element [c][l][i] at
 *    momenta[(c * n_ext + l) * n + i], c = 0..3 (E, px, py, pz) in GeV, l over the
 *    process legs in the order of the process name (two incoming legs first), i over
 *    the n points.  Points must be in the partonic centre-of-mass frame with the
 *    beams along +z (leg 0) and -z (leg 1) for the FKS entry points.
 *  - ps_weights: optional float64[n] (NULL = all 1) multiplied into each output.
 *  - out: float64[n].
 *  - pointers may be host (pageable or pinned) or device memory of the handle's
 *    device; the kind is detected per pointer.  Pinned (page-locked, mapped) host
 *    buffers are read and written by the kernels in place, over the coherent CPU-GPU
 *    link; pageable ones are copied through device scratch.  With any host pointer
 *    the call returns after the results are in `out`.  With device pointers only, the
 *    work is enqueued on the handle's stream and the call returns without
 *    synchronising (me_synchronize waits).
 *  - ownership: the caller owns all input and output buffers and keeps them alive
 *    until the results are ready; the library owns its handles, process tables and
 *    scratch, freed by me_destroy.
 *  - errors: every int-returning call returns ME_OK (0) or a negative ME_ERR_* code
 *    and sets a thread-local message readable with me_last_error(); no exception
 *    crosses the boundary.  A failed call leaves `out` unspecified.
 */
#ifndef ME_GB300_H
#define ME_GB300_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define ME_OK 0
#define ME_ERR_ARG (-1)      /* invalid argument (NULL handle, n < 0, bad sizes, bad params) */
#define ME_ERR_OOM (-2)      /* device or host allocation failed */
#define ME_ERR_PROCESS (-3)  /* unknown process or entry point not defined for it */
#define ME_ERR_TIMEOUT (-4)  /* a bounded wait ran out (me_poll) */
#define ME_ERR_CUDA (-5)     /* a CUDA call failed; see me_last_error() */
#define ME_ERR_BUSY (-6)     /* request rejected: queue full or over the memory budget */

#define ME_PARAMS_VERSION 4u
#define ME_PREC_FP64 0   /* every amplitude in float64 */
#define ME_PREC_MIXED 1  /* float32 amplitudes; float64 FKS maps, combination and rescue */
#define ME_RESCUE_POINTS 0 /* mixed precision: every flagged point re-evaluated whole in float64 */
#define ME_RESCUE_ITEMS 1  /* mixed precision: the flagged points' float64 items (see me_params) */
#define ME_TERMS_MASKED 0  /* subtracted real: Algorithm 2, every term evaluated, then masked */
#define ME_TERMS_QUEUED 1  /* subtracted real: per-term queues (see me_params) */
#define ME_TERMS_AUTO 2    /* queued for mixed-precision batches of at least 2^19 points, else masked */

/*
 * Run parameters.  Start from me_default_params(); `version` must equal
 * ME_PARAMS_VERSION.
 *   alpha, alpha_s   couplings (alpha_s fixed, renormalisation scale = sqrt(s))
 *   mt               top-quark mass [GeV]
 *   xi_cut, delta    FKS plus-distribution cut-offs xi_c in (0,1], delta in (0,2]
 *   xi_thr, y_thr    mixed mode: points with xi < xi_thr or 1-y < y_thr in an active
 *                    counterterm region are re-evaluated in float64
 *   tol, me_eps      mixed mode: a point is re-evaluated in float64 when
 *                    (E_R (1 + sqrt(0.01 / rho)) + E_B) me_eps > tol |W|, W = R S - CT
 *                    summed over sectors, E_R = sum over sectors of |R S|, E_B = sum
 *                    over sectors of |CT_coll| + |CT_soft - CT_softcoll| (the soft pair
 *                    shares its Born values, so their errors cancel), rho = min over
 *                    sectors of 1 - y (the float32 errors of the real's amplitudes grow
 *                    towards the collinear limit; the Born values at their regular 2 ->
 *                    2 kinematics do not); me_eps is
 *                    calibrated so that, with the flagged points re-evaluated, 99.9 %
 *                    of flat points of each real process stay within 0.7 tol (a 30 %
 *                    margin) and points on soft/collinear approach sequences within tol
 *   device           CUDA device ordinal the handle runs on
 *   lanes_per_event  lanes sharing one point (1, 2, 4, 8 or 16; at most 8 for
 *                    "gg_ttgg"; 0 = autotune: each candidate is timed once per device,
 *                    process, kind, precision and batch-size class floor(log2 n)
 *                    (capped at 15), on the first call that meets it, and the choice is
 *                    shared by every handle).  The queued mixed-precision subtracted real
 *                    always runs one lane per point.
 *   queued_rescue    mixed-precision subtracted real: 0 (default) = a float32 launch
 *                    that lists the unstable points, then a float64 launch over the
 *                    list; 1 = one launch in which each block queues its unstable
 *                    points in shared memory and re-evaluates them in float64
 *                    whenever the queue holds 128, next to other blocks' float32
 *                    work.  Both give the same results to float64 rounding; on GB300
 *                    the two launches are faster (the float64 unit needs several
 *                    warps per scheduler to stay busy).
 *   rescue           mixed-precision subtracted real with two launches (queued_rescue 0):
 *                    ME_RESCUE_ITEMS (default) re-evaluates, per flagged point, only the
 *                    ingredients whose float32 error the point cannot absorb.  The
 *                    subtracted weight is linear in its matrix-element ingredients --
 *                    the real's helicity blocks and the counterterms' Born values -- with
 *                    float64 coefficients from the FKS maps; a flagged point takes its
 *                    ingredients in float64, largest error scale first, until the
 *                    float32 error left is within tol |W| / 2, and W is recombined in
 *                    float64.  Points inside xi_thr / y_thr take every ingredient in
 *                    float64.  ME_RESCUE_POINTS re-evaluates every flagged point whole in
 *                    float64.  me_last_rescued counts the flagged points either way.
 *   term_queues      subtracted real (both precisions): ME_TERMS_MASKED = Algorithm 2 of the
 *                    paper (Sec. 4.3): every term -- real, soft, collinear -- is evaluated
 *                    for every point, and the terms whose cuts fail are zeroed afterwards;
 *                    ME_TERMS_QUEUED = per-term queues, the variant discussed after
 *                    Algorithm 2: a
 *                    float64 pass maps every point, decides the cuts and the counterterm
 *                    regions, and queues only the amplitudes a point needs (the real's
 *                    helicity blocks if the real passes its cuts; the soft Born set and
 *                    the collinear Born set if that counterterm is active and passes);
 *                    each kind of amplitude is then evaluated over its queue in one
 *                    launch, and the weight is recombined (mixed precision: with the same
 *                    stability test and float64 item rescue).  Tree-level entries
 *                    (me_eval_born, me_eval_nbody_nlo) queue the points that pass the cuts.
 *                    Results agree with ME_TERMS_MASKED to rounding.  ME_TERMS_AUTO
 *                    (default) takes the queues for mixed-precision batches of at least
 *                    2^19 points (on GB300 they are faster there, and slower on small
 *                    batches, whose extra launches and float64 pass do not amortise) and
 *                    the masked evaluation otherwise; queued_rescue 1 or rescue
 *                    ME_RESCUE_POINTS, options of the masked evaluation, select it.  With
 *                    ME_TERMS_QUEUED the queues always run their item rescue.  The allocation-free entry and the
 *                    persistent serving kernels always run the masked evaluation.
 *   cut_pt_min, cut_abs_y_max
 *                    cuts on both heavy quarks (legs 2, 3 of the t tbar processes and of
 *                    their Born counter-events): p_T >= cut_pt_min [GeV] and |rapidity
 *                    along the z axis| <= cut_abs_y_max.  0 and +infinity: no cut.
 *   cut_abs_cos_axis_max, cut_thrust_max
 *                    e+e- processes: |cos| of the thrust axis (the direction of the most
 *                    energetic final parton) with the z axis <= cut_abs_cos_axis_max, and
 *                    thrust T = max_i 2 E_i / sqrt(s) <= cut_thrust_max.  Values >= 1: no cut.
 *                    Each cut is applied to every term at that term's own kinematics (the
 *                    real point, or the soft or collinear Born counter-event); cuts that do
 *                    not belong to the handle's process are ignored.  Decisions are taken
 *                    in float64 without square roots or logarithms: px*px + py*py >=
 *                    pt_min^2, E + |pz| <= exp(2 y_max) (E - |pz|), pz^2 <= c^2 |p|^2,
 *                    2 E_m <= T_max (E_0 + E_1).
 */
typedef struct me_params {
  uint32_t version;
  int32_t precision;
  double alpha;
  double alpha_s;
  double mt;
  double xi_cut;
  double delta;
  double xi_thr;
  double y_thr;
  double tol;
  double me_eps;
  int32_t device;
  int32_t lanes_per_event;
  int32_t queued_rescue;
  int32_t rescue;
  int32_t term_queues;
  double cut_pt_min;
  double cut_abs_y_max;
  double cut_abs_cos_axis_max;
  double cut_thrust_max;
} me_params;

typedef struct me_handle me_handle;

/* Fill `p` with the defaults: FP64, alpha = 1/132.507, alpha_s = 0.118, mt = 173,
 * xi_cut = 0.5, delta = 1, xi_thr = 1e-3, y_thr = 1e-3, tol = 1e-5, me_eps = 4e-7,
 * device 0, lanes_per_event 0, queued_rescue 0, rescue ME_RESCUE_ITEMS, term_queues ME_TERMS_AUTO,
 * no cuts (cut_pt_min 0, cut_abs_y_max +infinity, cut_abs_cos_axis_max 1,
 * cut_thrust_max 1).  Never fails. */
void me_default_params(me_params* p);

/*
 * Create a handle for one process.  `process` is one of
 *   "ee_uu"   e+ e- -> u ubar          (legs e+, e-, u, ubar)
 *   "ee_uug"  e+ e- -> u ubar g        (legs e+, e-, u, ubar, g)
 *   "gg_tt"   g g -> t tbar            (legs g, g, t, tbar)
 *   "gg_ttg"  g g -> t tbar g          (legs g, g, t, tbar, g)
 *   "gg_ttgg" g g -> t tbar g g        (legs g, g, t, tbar, g, g)
 *   "uu_tt"   u ubar -> t tbar         (legs u, ubar, t, tbar)
 *   "uu_ttg"  u ubar -> t tbar g       (legs u, ubar, t, tbar, g)
 * Sets up the device-resident process constants (colour matrices, colour
 * correlators, couplings) on `params->device` on first use of that device.
 * Returns ME_ERR_PROCESS for an unknown name, ME_ERR_ARG for bad params.
 */
int me_init(const char* process, const me_params* params, me_handle** out);

/* Number of legs of the handle's process (for sizing momentum buffers). */
int me_n_external(const me_handle* h);

/*
 * Tree-level squared matrix element (Sec. 2.1, Eq. (born); Sec. 2.2, Eq. (real)),
 * summed over helicities and colours, averaged over initial spins and colours, with
 * the identical-final-particle factor:  out[i] = ps_weights[i] * |M|^2(p_i).
 * Defined for every process.  Adds (sum out, sum out^2, n) to the accumulators.
 */
int me_eval_born(me_handle* h, const double* momenta, const double* ps_weights, int64_t n, double* out);

/*
 * n-body NLO weight of e+e- -> u ubar: Born + virtual + integrated FKS
 * counterterms, out[i] = ps_weights[i] * B_i * (1 + a_s (5 - 2 pi^2/3
 * - (3 + 4 ln xi_cut) ln(delta/2))), a_s = alpha_s C_F / (2 pi).  Only "ee_uu".
 */
int me_eval_nbody_nlo(me_handle* h, const double* momenta, const double* ps_weights, int64_t n, double* out);

/*
 * Real-emission weight minus FKS soft and collinear counterterms, summed over the FKS
 * sectors (Sec. 2.2: FKS subtraction; Sec. 4.2: one kinematic parametrisation per
 * sector; Sec. 4.3, Algorithm 2: every term computed, then masked by the cut-offs):
 *   out[i] = ps_weights[i] * sum_j [ R S_j - (Th_s G(0,y) + Th_c G(xi,1)
 *                                    - Th_s Th_c G(0,1)) / (xi^2 (1-y) K) ].
 * Defined for "ee_uug" (final-state sectors) and "gg_ttg", "uu_ttg" (initial-state
 * sectors).  In ME_PREC_MIXED, points failing the stability test are recomputed in
 * float64 before the call's results are complete.  Points on the boundary of the FKS
 * domain (xi = 0 or 1, or the emission exactly along a sector's reference direction)
 * have measure zero and no defined subtracted weight: out[i] = 0 for them.  Adds to the
 * accumulators.
 */
int me_eval_real_subtracted(me_handle* h, const double* momenta, const double* ps_weights, int64_t n, double* out);

/* Number of points re-evaluated in float64 by the last me_eval_real_subtracted call
 * (synchronises the handle's stream). */
int me_last_rescued(me_handle* h, int64_t* n_rescued);

/* Float64 work of the last me_eval_real_subtracted call in mixed precision with the item
 * rescue: the flagged points, the real-emission helicity blocks and the sets of
 * counterterm Born values re-evaluated in float64 (with ME_RESCUE_POINTS or the queued
 * kernel only the points are counted; the other two are 0).  With the per-term queues
 * (me_params.term_queues) born_sets counts Born configurations, soft and collinear
 * separately.  Synchronises the handle's stream. */
int me_last_rescue_work(me_handle* h, int64_t* points, int64_t* real_blocks, int64_t* born_sets);

/* The float64 Born configurations of the last mixed-precision me_eval_real_subtracted
 * call that ran the per-term queues (Sec. 4.3), by kind: set0 = soft counter-events
 * (initial state) or sector-1 Borns (final state), set1 = collinear counter-events or
 * sector-2 Borns.  Both 0 after a call that ran the masked evaluation.  Synchronises
 * the handle's stream. */
int me_last_rescue_configs(me_handle* h, int64_t* set0, int64_t* set1);

/* Monte-Carlo accumulators of all outputs since creation or the last set:
 * out[0] = sum w, out[1] = sum w^2, out[2] = number of points (as double).
 * Synchronises the handle's stream.  me_set_accumulators restores them (resume). */
int me_get_accumulators(me_handle* h, double out[3]);
int me_set_accumulators(me_handle* h, const double in[3]);

/* Stage timers (profiling, off by default).  When enabled, every evaluation records
 * CUDA events on the handle's stream around its main kernel, its float64 rescue
 * kernel and its weight reduction (at most 4096 calls are kept).  me_stage_times
 * synchronises, returns the summed durations in milliseconds (out_ms[0] main kernel,
 * [1] rescue, [2] reduction) and the number of timed calls, and clears them. */
int me_enable_stage_timers(me_handle* h, int on);
int me_stage_times(me_handle* h, double out_ms[3], int64_t* calls);

/* Use an existing cudaStream_t (passed as void*) for the handle's work; NULL selects
 * the handle's own stream.  The caller keeps the stream alive while it is in use. */
int me_set_stream(me_handle* h, void* cuda_stream);

/* Wait until all work enqueued on the handle's stream has finished. */
int me_synchronize(me_handle* h);

/* Flat phase-space points of the handle's process generated on the device (the
 * multi-event input of Sec. 4.4 produced where it is evaluated): points first_point ..
 * first_point + n - 1 of the counter-based stream (seed, stream) -- Philox4x32-10 with
 * counter (point lo, point hi, stream, block) and key (seed lo, seed hi), uniforms
 * ((w0 >> 5) 2^26 + (w1 >> 6) + 1/2) 2^-53 -- turned into momenta by RAMBO (massless
 * directions and energies -log(u u'), boosted and scaled to sqrt_s) with the massive
 * rescaling for the top quarks (mass params.mt).  Beams: massless along +z and -z.
 * momenta: device float64 [4][n_ext][n] (layout as above); ps_weights: device float64[n]
 * (the phase-space weight of each point) or NULL.  Enqueued on the handle's stream.
 * ME_ERR_ARG for host pointers, n < 0 or sqrt_s not above the final-state masses. */
int me_generate_flat(me_handle* h, uint64_t seed, uint32_t stream, int64_t first_point, double sqrt_s, int64_t n,
                     double* momenta, double* ps_weights);

/* Phase-space points of a real-emission process ("ee_uug", "gg_ttg", "uu_ttg") generated
 * on the device directly in the variables of its FKS sectors (Sec. 4.2: each sector has
 * its own kinematic parametrisation), with a density that samples the soft and collinear
 * regions the subtraction has to handle: the emitted gluon's energy fraction xi flat
 * (flat three-body phase space has density ~ xi there), its cosine y_j w.r.t. the
 * sector's reference direction as y_j = 1 - 2 v^2 with v uniform (density
 * 1 / (4 sqrt((1 - y_j)/2))), azimuth and Born direction uniform; the two sectors are
 * channels of one multichannel density, and each weight is the phase-space measure over
 * the summed density.  Uniforms u0..u5 of point i: Philox4x32-10 blocks 0..2 at counter
 * (i lo, i hi, stream, block), key (seed lo, seed hi), mapped as in me_generate_flat.
 *   initial-state sectors (gg_ttg, uu_ttg): xi = (1 - 4 mt^2/s) u0, y_j = 1 - 2 u1^2 w.r.t.
 *     beam j (j = 0 along +z if u5 < 1/2, else the -z beam), phi = 2 pi u2, the heavy
 *     pair's rest-frame direction (cos 2 u3 - 1, azimuth 2 pi u4);
 *   final-state sectors (ee_uug): partner leg 2 if u0 < 1/2 else leg 3, its direction
 *     (cos 2 u1 - 1, azimuth 2 pi u2), xi = u3, y_j = 1 - 2 u4^2, phi = 2 pi u5 about it.
 * Layout, beams, device buffers and errors as for me_generate_flat; ME_ERR_PROCESS for a
 * process without FKS sectors.  Enqueued on the handle's stream. */
int me_generate_fks(me_handle* h, uint64_t seed, uint32_t stream, int64_t first_point, double sqrt_s, int64_t n,
                    double* momenta, double* ps_weights);

/*
 * Unweighted events from weighted points: the accept/reject step that turns a sample
 * weighted by the integrand into events distributed like it (Sec. 3.1), for signed NLO
 * weights.  Point i is kept iff u_i * w_max < |w_i|, where u_i in (0,1) is the first
 * uniform of Philox4x32-10 (key = seed) at counter (lo and hi words of first_point + i,
 * stream, 0), mapped as in me_generate_flat: ((x0 >> 5) 2^26 + (x1 >> 6) + 1/2) 2^-53.
 * A kept point carries the event weight sign(w_i) * max(w_max, |w_i|), so the expected
 * event weight of every point is w_i; points with |w_i| > w_max (overweight) are always
 * kept with their own weight.  Use a `stream` other than the one that generated the
 * points.  NaN weights are never kept.
 *   weights       device float64[n]
 *   w_max         > 0: used as given; <= 0: the maximum of |w_i| over the batch
 *   kept          device int32[n]: the indices of the kept points, in increasing order
 *   kept_weights  device float64[n] or NULL: their event weights
 *   n_kept        host: number of kept points (entries written to kept, kept_weights)
 *   w_max_used    host or NULL: the w_max applied
 *   n_over        host or NULL: number of overweight points (all kept)
 * Runs on the handle's stream and returns when the results are in place.  ME_ERR_ARG for
 * host buffers, n outside [0, 2^31), first_point < 0 or a NaN w_max.
 */
int me_unweight(me_handle* h, const double* weights, int64_t n, double w_max, uint64_t seed, uint32_t stream,
                int64_t first_point, int32_t* kept, double* kept_weights, int64_t* n_kept, double* w_max_used,
                int64_t* n_over);

/* Release the handle and its device scratch (waits for its stream).  NULL is a no-op. */
void me_destroy(me_handle* h);

/* ---------------------------------------------------------------- request loop
 * Continuous batching of phase-space batches from many integration channels
 * (the multi-event interface of Sec. 4.4; points stay on the device for the whole
 * evaluation, Sec. 4.3).  A server owns `n_slots` slots on one device, each a host
 * thread with its own CUDA stream; a free slot admits the oldest queued request
 * whenever the sum of the in-flight requests' buffers (n * (4 n_ext + 2) * 8 bytes)
 * stays within `mem_budget_bytes`, so requests that arrive while others run are
 * admitted as slots and memory free up, and their staging and kernels overlap.  A
 * request's result does not depend on what else is in flight.
 */
#define ME_KIND_BORN 0             /* me_eval_born */
#define ME_KIND_REAL_SUBTRACTED 1  /* me_eval_real_subtracted */
#define ME_KIND_NBODY_NLO 2        /* me_eval_nbody_nlo */

typedef struct me_server me_server;
typedef uint64_t me_ticket;

typedef struct me_server_params {
  uint32_t version;          /* ME_PARAMS_VERSION */
  int32_t device;            /* CUDA device ordinal */
  int32_t n_slots;           /* concurrent requests on the device, 1..64 */
  int32_t max_queue;         /* pending requests beyond which me_submit returns ME_ERR_BUSY */
  int64_t mem_budget_bytes;  /* admission budget for in-flight request buffers */
  me_params params;          /* physics and precision, shared by all requests */
  int32_t use_graphs;        /* 1: replay each (process, kind) launch sequence from a captured CUDA graph */
  int32_t persistent;        /* 1: the e+e-, g g and u ubar families (ee_uu/ee_uug, gg_tt/gg_ttg,
                                uu_tt/uu_ttg) run on one persistent kernel per family that reads
                                work descriptors from a ring in pinned host memory (no launch
                                per request); gg_ttgg stays on the slots */
  int32_t persistent_idle_us; /* a persistent kernel with no work for this long ends with
                                 ME_ERR_TIMEOUT (counted by me_server_persistent_stats) and is
                                 launched again by the next request of its family */
} me_server_params;

/* One batch: host buffers owned by the caller, kept alive until me_poll returns it. */
typedef struct me_request {
  const char* process;       /* process name as for me_init */
  int32_t kind;              /* ME_KIND_* */
  const double* momenta;     /* host, [4][n_ext][n] as above */
  const double* ps_weights;  /* host float64[n] or NULL */
  int64_t n;
  double* out;               /* host float64[n], written before me_poll reports it */
} me_request;

typedef struct me_result {
  int32_t status;            /* ME_OK or the ME_ERR_* code of the evaluation */
  int64_t n;
  int64_t n_rescued;         /* points re-evaluated in float64 (mixed precision) */
  double sum_w, sum_w2;      /* of out[] */
  double t_queue_us;         /* submit -> admission */
  double t_device_us;        /* copies + kernels on the slot's stream (CUDA events) */
  double t_total_us;         /* submit -> completion seen by the slot thread */
} me_result;

/* Defaults: device 0, 4 slots, queue 4096, 8 GiB budget, mixed precision, graphs on,
 * persistent kernels off (idle limit 2000 us when on). */
void me_default_server_params(me_server_params* p);
/* Start a server and its slot threads.  ME_ERR_ARG for bad parameters. */
int me_server_create(const me_server_params* params, me_server** out);
/* Queue a request; returns a ticket.  ME_ERR_BUSY when the queue is full or the
 * request alone exceeds the memory budget; ME_ERR_PROCESS for an unknown process. */
int me_submit(me_server* s, const me_request* req, me_ticket* out);
/* Wait up to timeout_us (negative: no limit) for a ticket.  ME_OK: `out` filled and
 * the ticket retired; ME_ERR_TIMEOUT: not finished yet (poll again); ME_ERR_ARG:
 * unknown or already retired ticket.  The wait is on the host only. */
int me_poll(me_server* s, me_ticket t, me_result* out, int64_t timeout_us);
/* Requests run so far by replaying a captured CUDA graph (every request of a
 * (process, kind, weights) key after the first on a slot) and by ordinary launches. */
int me_server_stats(me_server* s, int64_t* graph_runs, int64_t* plain_runs);
/* Persistent kernels (server created with persistent = 1), summed over the families:
 * kernel launches, launches that ended because their wait for work ran out
 * (ME_ERR_TIMEOUT, the idle limit), and requests served by them.  The wait is a bounded
 * device-side poll of the descriptor ring; every other wait in those kernels is bounded
 * too, so a kernel always ends. */
int me_server_persistent_stats(me_server* s, int64_t* launches, int64_t* idle_timeouts, int64_t* requests);
/* Stop the slot threads, wait for in-flight work, free everything.  NULL is a no-op. */
void me_server_destroy(me_server* s);

/* ---------------------------------------------------------------- allocation-free variant
 * The paper has no counterpart to this entry point.  It serves callers that cannot
 * allocate GPU memory: code whose device memory belongs entirely to another allocator
 * (for example a host application's caching pool), code that must not trigger the
 * device-wide synchronisation that cudaMalloc and cudaFree imply, and code running
 * where allocation is not permitted.
 *
 * Same weights as me_eval_real_subtracted ("ee_uug", "gg_ttg", "uu_ttg"), without a
 * handle and without any allocation (no cudaMalloc, cudaFree or other allocating call).
 * Its only scratch is a built-in device array -- the mixed-precision rescue list and
 * its counter, (ME_NOALLOC_MAX_POINTS + 64) int32 = 4 MiB -- that every GPU loading the
 * library holds until the process exits; the process tables live in a second built-in
 * device object.
 *  - momenta, ps_weights (optional) and out must be device memory of params->device;
 *    n larger than ME_NOALLOC_MAX_POINTS is rejected with ME_ERR_ARG.
 *  - the work is enqueued on `cuda_stream` (NULL: the legacy default stream) and the call
 *    returns without waiting; results are ready when that stream reaches this point.
 *  - the first call on a device sets the device up (looks up the built-in arrays'
 *    device addresses and uploads the process tables, synchronously); make that first
 *    call before any stream capture.
 *  - all calls share the built-in scratch, which keeps the last call's contents; each
 *    call clears the rescue counter on its stream before use.  Calls whose work overlaps
 *    on the GPU (other streams, other threads) race on the scratch: serialise them.
 *  - lanes_per_event 0 selects 4 (no autotuning); the accumulators are not touched.
 */
#define ME_NOALLOC_MAX_POINTS 1048576
int me_eval_real_subtracted_noalloc(const char* process, const me_params* params, const double* momenta,
                                    const double* ps_weights, int64_t n, double* out, void* cuda_stream);

/* Message of the last failed call on this thread ("" if none).  Valid until the next
 * call on the same thread. */
const char* me_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* ME_GB300_H */
