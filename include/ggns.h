/*
 * ggns.h -- C ABI of the GB300 (sm_103a) gradient-guided nested sampling library.
 *
 * The library runs the data-parallel hot path of gradient-guided nested sampling
 * (GGNS, arXiv 2312.03911) on one GPU: batched Hamiltonian slice sampling of all
 * replacement points at once (Algorithm 5), fused log-likelihood and score
 * evaluation, reflection p' = p - 2 (p.n) n (Section 2.3), step-size adaptation
 * (Algorithm 3), lowest-likelihood selection, k-NN cluster finding (Algorithm 4),
 * the FP64 cluster statistics of Appendix H and the evidence
 * Z = int L(theta) pi(theta) dtheta (Section 2.1) with its error.
 *
 * Conventions for every call:
 *   - Return value: NS_OK or an error status; nothing throws or aborts across
 *     the ABI.  ns_last_error() describes the last failure of a context.
 *   - Input arrays are owned by the caller and copied before the call returns.
 *   - Pointers named *_dev are device pointers (CUDA global memory of the current
 *     device); all others are host pointers.
 *   - Work is queued on the context's stream (ns_set_stream; default: the legacy
 *     default stream); calls that return host data synchronise that stream.
 *   - Floating-point inputs arrive in FP64; the walkers compute in FP32 and the
 *     evidence statistics in FP64.
 *   - A device-side failure (capacity exhausted, no finite likelihood) is stored
 *     in the run's status word and returned by the next call that reads it.
 */
#ifndef GGNS_H
#define GGNS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct ns_ctx ns_ctx; /* opaque; created by ns_create / ns_batch_create */

typedef enum {
    NS_OK = 0,
    NS_ERR_ARG = 1,      /* invalid argument (NULL, out-of-range size or option)        */
    NS_ERR_CUDA = 2,     /* a CUDA runtime call failed; see ns_last_error              */
    NS_ERR_OOM = 3,      /* device allocation failed                                    */
    NS_ERR_TIMEOUT = 4,  /* a bounded device loop hit its iteration limit               */
    NS_ERR_STUCK = 5,    /* reserved: walkers could not leave an empty slice            */
    NS_ERR_NUMERIC = 6,  /* no live point has a finite log-likelihood                   */
    NS_ERR_NOT_DONE = 7, /* the run stopped at max_iters before its termination test    */
    NS_ERR_CAPACITY = 8, /* dead-point arena, cluster table or output buffer too small  */
    NS_ERR_BOUNDS = 9    /* checked builds only (GGNS_CHECKED): an index check of the   */
                         /* dead-point arena, the step records or the live slots failed */
} ns_status;

typedef enum {
    NS_LIK_ISO_GAUSS = 0,   /* N(x; mu, sigma^2 I), normalised                           */
    NS_LIK_MIX_ISO = 1,     /* sum_k w_k N(x; mu_k, sigma_k^2 I)                          */
    NS_LIK_DENSE_GAUSS = 2, /* N(x; mu, P^-1) with precision P                            */
    NS_LIK_DENSE_MIX = 3,   /* sum_k w_k N(x; mu_k, P^-1), one precision for all          */
    NS_LIK_ROSENBROCK = 4,  /* -scale * sum_i [100 (x_{i+1} - x_i^2)^2 + (1 - x_i)^2]     */
    NS_LIK_TORUS = 5        /* the torus reward of Section 4, eq. torus (see below)      */
} ns_lik_kind;

/* Uniform prior on the box [lo_i, hi_i] (the prior pi of Section 2.1). */
typedef struct {
    int d;
    const double *lo; /* [d] */
    const double *hi; /* [d] */
} ns_prior_box;

/* Likelihood family and parameters (the L(theta) of Section 2.1). */
typedef struct {
    ns_lik_kind kind;
    int d;
    int n_comp;                /* components; 1 for the single-Gaussian kinds            */
    const double *means;       /* [n_comp][d] row-major (unused by ROSENBROCK)           */
    const double *log_weights; /* [n_comp] log mixture weights, NULL = equal weights     */
    const double *sigma;       /* [n_comp] isotropic standard deviations (ISO kinds)     */
    const double *precision;   /* [d][d] row-major symmetric positive definite (DENSE)   */
    double rosen_scale;        /* ROSENBROCK multiplier (1/20 for the benchmark)         */
    /* TORUS (Section 4, eq. torus; Appendix F): L = (sum of sin(torus_alpha x_i) over the
     * even 1-based coordinates x_2, x_4, ... + sum of cos(torus_beta x_j) over the odd ones
     * x_1, x_3, ... + torus_c)^3.  torus_c > d keeps L > 0; integer frequencies make the
     * normaliser of Appendix F exact.  The prior box of a TORUS run is a torus: a walker
     * step wraps every coordinate into [lo_i, hi_i) and never leaves the prior.  means,
     * sigma, precision and log_weights are unused. */
    double torus_alpha, torus_beta, torus_c;
} ns_likelihood_spec;

/* Sampler hyper-parameters (Appendix C table; Algorithms 3 and 5). */
typedef struct {
    int n_live;        /* live points; n_live/2 are killed and replaced per iteration (Section 3) */
    int n_steps;       /* hard cap on HSS steps per iteration                                    */
    int min_steps;     /* HSS runs at least this many steps                                       */
    double dt_init;    /* initial step size dt_ini                                                */
    double delta_p;    /* momentum noise amplitude                                                */
    double tol;        /* termination tolerance                                                   */
    int min_ref;       /* inside states are saved once every walker reflected min_ref times      */
    int max_ref;       /* HSS stops once every walker reflected max_ref times                     */
    int prune_after;   /* consecutive outside steps after which a walker restarts (0 = never)    */
    int termination;   /* 0: XL-peak L_i X_i / max L_i X_i < tol; 1: X L_max < tol Z             */
    int clustering;    /* 1: cluster finding of Algorithm 4 every iteration                       */
    int noise_mode;    /* 0: p *= 1 + delta_p eps (as printed); 1: p = sqrt(1-dp^2) p + dp eps   */
    double out_lo;     /* dt *= 1.1 when out_frac < out_lo (0.05 in Algorithm 3)                  */
    double out_hi;     /* dt *= 0.9 when out_frac > out_hi (0.15 in Algorithm 3)                  */
    uint64_t seed;     /* Philox key; run r of a batch uses key (seed_lo, seed_hi ^ run_id)      */
    uint32_t run_id;   /* first run id; run r of a batch uses run_id + r                          */
    long max_iters;    /* iteration cap                                                           */
    long dead_cap;     /* dead-point arena capacity per run; 0 = estimate from d and tol          */
    /* Readings of Algorithm 5 and of the cluster bookkeeping of Algorithm 3 (Section 2.3,
     * Section 3).  1 in each selects the form the library defaults to; 0 the printed form. */
    int noise_inside;  /* 1: the momentum noise perturbs inside steps only, an outside step only
                          reflects (Section 2.3: a particle can get stuck behind the boundary)
                          0: every step takes the noise, as Algorithm 5 prints it                */
    int pick_all;      /* 1: each walker returns a state drawn uniformly over every step of the
                          saving window; a drawn outside step is rejected and the walker returns
                          its start point (slice-sampling rejection, Section 2.3)
                          0: drawn uniformly over the saved inside states only (Algorithm 5)     */
    int territory;     /* 1: with several clusters alive, a new point whose nearest surviving
                          point belongs to another cluster returns its start point               */
    int keep_last;     /* Appendix G ablation: 1 returns the last inside state of the window
                          (with midpoint: the last state, tested against L* like any pick)      */
    int box_fold;      /* 0: leaving the prior box is an outside step, reflected off the violated faces
                          1: the box reflects a walker exactly (its position folds back across the
                          face, that momentum component flips; no outside step), so only the
                          iso-likelihood boundary of Algorithm 5 counts as outside              */
    int fold_counts;   /* with box_fold 1: 1 counts an inside step on which the box reflected the
                          walker as a reflection for the adaptive step size (Section 3: dt follows
                          the number of reflections); it never counts toward n_ref or the pick  */
    /* Launch choices; 0 selects the library's own choice.  Options marked (context) are read
     * from the first configuration of a batch; tile from the first run of each (kind, d).    */
    int tile;          /* walker tile id + 1: 1..N_TILES (G lanes x E components, ns_tile_shape) */
    int hss_mode;      /* (context) 1: single pass where resident; 2: three phases always        */
    int rec_len;       /* (context) step records per walker of the single pass (0: n_steps)     */
    int noise_ahead;   /* (context) steps of momentum noise drawn ahead (0: 128; -1: none)       */
    int coop;          /* (context) dense walk, 16 walkers per CTA sharing each read of P: 0 with
                          the contraction on the tensor cores where d_pad is 128, 256 or 512,
                          else on CUDA cores; 1 on CUDA cores; -1 off (one read per walker)     */
    int runs_per_group;/* (context) runs per concurrent group and graph (0: all in one group)    */
    /* The time-reversible form of Algorithm 5's step (an option; 0 keeps the step as printed):
     * half move, reflection with the normal at the half step if that point is outside, half
     * move; the refresh noise acts on every state; every step's state is recorded and the
     * state the pick draws is tested against L* afterwards (outside: the start point).  The
     * printed step (move, then reflect at the new point) is not time-reversible, and at high
     * d its evidence offset grows with the trajectory length.  Needs box_fold 1, noise_mode 1,
     * a non-periodic kind and the single-pass walk with records for every step (NS_ERR_ARG
     * otherwise).  With keep_last 1, min_ref 0, max_ref out of reach, min_steps = n_steps = K
     * and prune_after 0, every walker follows a reversible trajectory of exactly K steps and
     * returns its end point when inside, else its start point: an exact slice-sampling move
     * (a refresh p <- a p + b e with a^2 + b^2 = 1 is an orthogonal map of (p, e), so the
     * trajectory with the momentum flipped at its end is a measure-preserving involution),
     * whereas a window that opens and closes on the walkers' reflection counts is not. */
    int midpoint;
} ns_config;

/* Fills the defaults: n_live 200, n_steps 1000, min_steps 0, dt_init 0.1,
 * delta_p 0.5, tol 0.01, min_ref 1, max_ref 3, prune_after 10, termination 0,
 * clustering 1, noise_mode 1, out_lo 0.05, out_hi 0.15, seed 0, run_id 0,
 * max_iters 100000, dead_cap 0, noise_inside 1, pick_all 1, territory 1,
 * keep_last 0, box_fold 0, fold_counts 0, every launch choice 0 (the library's own) and
 * midpoint 0. */
void ns_config_default(ns_config *cfg);

/* Create a context for one run.  Copies the box, the likelihood parameters and
 * the configuration to the device, draws the n_live prior points (Algorithm 3,
 * first step) and evaluates them.  *out receives a context owned by the caller
 * (free with ns_destroy).  Errors: NS_ERR_ARG for inconsistent sizes, d < 1,
 * n_live < 2 or > 16384, n_comp outside [1, 64], min_ref > max_ref, a
 * precision that is not positive definite; NS_ERR_OOM; NS_ERR_CUDA. */
ns_status ns_create(const ns_prior_box *box, const ns_likelihood_spec *lik, const ns_config *cfg,
                    ns_ctx **out);

/* Create one context holding n_runs independent runs (box[r], lik[r], cfg[r]
 * for r = 0..n_runs-1), advanced together: every kernel of an iteration covers
 * all runs, finished runs idle.  Same errors as ns_create. */
ns_status ns_batch_create(int n_runs, const ns_prior_box *box, const ns_likelihood_spec *lik,
                          const ns_config *cfg, ns_ctx **out);

/* Queue all later work of ctx on `cuda_stream` (a cudaStream_t, e.g. torch's
 * current stream).  NULL selects the legacy default stream. */
ns_status ns_set_stream(ns_ctx *ctx, void *cuda_stream);

/* Advance every unfinished run by up to n_iters iterations of Algorithm 3.
 * *done (may be NULL) receives 1 when every run has met its termination test
 * or its iteration cap.  Synchronises the stream once at the end. */
ns_status ns_step(ns_ctx *ctx, int n_iters, int *done);

/* Run until every run terminates (or max_iters), then perform the final sweep
 * of the remaining live points (Algorithm 3, last loop).  Iterations are
 * replayed as CUDA graphs of several iterations each; the host reads the
 * termination flags once per graph. */
ns_status ns_run(ns_ctx *ctx, long max_iters);

/* Start every run of ctx again from a fresh prior draw with Philox seed `seed`
 * (run r keys its stream with (seed_lo, seed_hi ^ run_id_r)), keeping all
 * allocations: statistics, counters and dead points are reset on the device.
 * Used to repeat a workload without allocating.  Synchronises. */
ns_status ns_restart(ns_ctx *ctx, uint64_t seed);

/* Profiling counters of ctx (out[10]): out[0] milliseconds during which at
 * least one HSS kernel of ns_run was executing (union over the run groups of
 * the intervals between CUDA events recorded around the HSS kernels of each
 * iteration), out[1] group-iterations measured, out[2] kernels launched by
 * ctx, out[3] rounds of graph replays, out[4] the summed (not merged) HSS
 * intervals, out[5] iterations (summed over runs, since the last restart) whose
 * single-pass HSS ran out of step records and was redone in three phases,
 * out[6] step records per walker (0: the three-phase form only), out[7] steps
 * of momentum noise drawn ahead per walker (0: drawn during the walk), out[8]
 * walker classes stepping CTA-cooperatively (dense likelihoods whose precision
 * matrix is read from global memory in shared tiles), out[9] those of them whose
 * contraction runs on the tensor cores (tcgen05 kind::f16, a scaled two-term FP16 split).
 * reset != 0 zeroes out[0..4] after reading.  Synchronises. */
ns_status ns_profile(const ns_ctx *ctx, double *out, int reset);

typedef struct {
    double logz;              /* log of the FP64 mean evidence Zbar (Appendix H)              */
    double logz_err;          /* sqrt(log Z^2bar - 2 log Zbar), moment-matched log-normal      */
    double logz_skilling_err; /* sqrt(H / n_live), eq. for sigma(log Z) in Section 2.1        */
    double info_h;            /* H = sum_i p_i log(L_i / Z), p_i the posterior weights          */
    long n_iter;              /* iterations of Algorithm 3                                     */
    long n_dead;              /* dead points, final sweep included                             */
    long n_like;              /* likelihood evaluations (prior draws + HSS point-steps)        */
    long n_steps_total;       /* HSS point-steps                                               */
    double dt;                /* final step size                                               */
    int n_clusters;           /* live clusters before the final sweep                          */
    int max_clusters;         /* largest number of clusters seen                               */
    int terminated;           /* 1 if the termination test fired                               */
    int status;               /* ns_status of the run                                          */
} ns_result_t;

/* Result of run 0 (or of run `run` with ns_result_run).  Synchronises. */
ns_status ns_result(const ns_ctx *ctx, ns_result_t *out);
ns_status ns_result_run(const ns_ctx *ctx, int run, ns_result_t *out);

/* Weighted posterior samples of run `run` (Appendix A, importance weights
 * p_i = L_i w_i / Z): x[cap][d] row-major and log p_i (normalised so that
 * sum_i p_i = 1).  With x == NULL and cap == 0 only *n_out (the number of dead
 * points) is written.  NS_ERR_CAPACITY if cap < n_out. */
ns_status ns_samples(const ns_ctx *ctx, int run, double *x, double *logp, long cap, long *n_out);

/* d log Z / d mu_k for every component mean of run `run`: the posterior-
 * weighted average sum_i p_i d log L(x_i) / d mu_k over the dead points, the
 * weights held fixed (from Z = int L pi, Section 2.1).  grad[n_comp][d];
 * NS_ERR_CAPACITY if cap < n_comp * d; NS_ERR_ARG for ROSENBROCK and TORUS (no means). */
ns_status ns_grad_logz(const ns_ctx *ctx, int run, double *grad, long cap);

/* Serialise / restore the complete sampler state (live set, statistics, step
 * size, counters, dead arena) so that a resumed run continues bit-identically;
 * the Philox counters depend only on (seed, run, iteration).  ns_state_save
 * with buf == NULL writes the required size to *n. */
ns_status ns_state_save(const ns_ctx *ctx, void *buf, size_t cap, size_t *n);
ns_status ns_state_load(ns_ctx *ctx, const void *buf, size_t n);

/* Description of the last error of ctx (a string owned by ctx), or of the
 * last failed ns_create when ctx is NULL. */
const char *ns_last_error(const ns_ctx *ctx);

/* Release every device and host resource of ctx. */
void ns_destroy(ns_ctx *ctx);

/* ------------------------------------------------------------------------ */
/* Component entry points: single steps of the hot path on caller data, used  */
/* by the parity tests.  All pointers are device pointers unless named *_host.*/
/* They run on `stream` (a cudaStream_t, NULL = default) and synchronise it.  */
/* ------------------------------------------------------------------------ */

/* Philox4x32-10 (Salmon et al., SC'11): out_dev[n][4] receives the words for
 * counters ctr_dev[n][4] under key (key0, key1). */
ns_status ns_philox(const uint32_t *ctr_dev, uint32_t key0, uint32_t key1, uint32_t *out_dev, long n,
                    void *stream);

/* log L and its gradient for n points x_dev[n][d] (row-major, FP32):
 * logl_dev[n], grad_dev[n][d] (grad_dev may be NULL).  The likelihood is the
 * one of run 0 of ctx.  This is the fused forward used by the walkers. */
ns_status ns_lik_forward(const ns_ctx *ctx, const float *x_dev, long n, float *logl_dev, float *grad_dev,
                         void *stream);

/* Replace the component means of run `run` by means_host[n_comp][d] (FP64,
 * row-major; copied before return): the parameters theta of the likelihood
 * whose log Z gradient the paper's problem statement asks for (Section 2.1).
 * ns_lik_forward / ns_lik_backward use them at once; sampling uses them after
 * ns_restart.  NS_ERR_ARG for ROSENBROCK and TORUS (no means).  Synchronises. */
ns_status ns_set_means(ns_ctx *ctx, int run, const double *means_host);

/* Adjoint of ns_lik_forward: given gout_dev[n] = d(loss)/d(log L_i),
 * gx_dev[n][d] = gout_i * d log L_i / dx_i and gmu_dev[n_comp][d] =
 * sum_i gout_i d log L_i / d mu_k (either output may be NULL; gmu_dev must be
 * NULL for ROSENBROCK and TORUS, which have no means: NS_ERR_ARG otherwise). */
ns_status ns_lik_backward(const ns_ctx *ctx, const float *x_dev, long n, const float *gout_dev,
                          float *gx_dev, float *gmu_dev, void *stream);

/* Algorithm 5 on caller data for run 0 of ctx: n walkers start at x0_dev[n][d]
 * (FP32, all inside L > lstar) with step dt at iteration `iter`; walker j uses
 * Philox slot j.  Writes the new points x_out_dev[n][d], logl_out_dev[n], the
 * per-walker step counts steps_dev[n] (may be NULL) and, in stats_host[5],
 * (n_in, n_out, t_save, t_stop, n_fold): inside and outside steps, the first
 * saving step, the last step, and the inside steps on which the box reflected a
 * walker (box_fold). */
ns_status ns_hss(const ns_ctx *ctx, const float *x0_dev, const float *logl0_dev, long n, float lstar,
                 double dt, uint32_t iter, float *x_out_dev, float *logl_out_dev, int *steps_dev,
                 long *stats_host, void *stream);

/* Algorithm 4 on m points x_dev[m][d] (FP32): comp_dev[m] receives the
 * smallest member index of each point's k-NN component; *n_comp_host the
 * number of components.  m <= 16384. */
ns_status ns_knn_components(const float *x_dev, int m, int d, int *comp_dev, int *n_comp_host,
                            void *stream);

/* Allocation-free form of ns_knn_components, for callers that cannot allocate
 * device memory when they run it (a host framework that owns all device memory
 * through its own pool, or a process whose device-memory budget is fixed at
 * start time).  The paper has no counterpart: this is an interface variant.
 * Same inputs, outputs and results as ns_knn_components, for m <= 4096 points
 * and d <= 512; larger m returns NS_ERR_ARG with a message in
 * ns_last_error(NULL).  Its scratch is one static device array (about 304 KiB)
 * that every GPU loading the library holds until the process exits; the call
 * allocates and frees nothing.  The first call on a device, with that device
 * current, looks up the array's device address; make that first call before
 * any stream capture.  The address is kept per driver context: after a device
 * reset (or any new primary context) the next call looks it up again, so that
 * call too should come before any stream capture.  Every call reuses the same array and leaves its contents
 * behind (each call re-initialises what it reads), so calls that overlap on the
 * GPU -- on different streams or host threads -- race and must be serialised
 * by the caller.  Synchronises `stream`. */
ns_status ns_knn_components_noalloc(const float *x_dev, int m, int d, int *comp_dev, int *n_comp_host,
                                    void *stream);

/* The region rule of the cluster bookkeeping (Algorithm 3 spawns a new point in
 * cluster p from one of p's survivors; Appendix H's statistics hold when a
 * cluster's live points stay in its region): keep_dev[j] = 1 when the nearest of
 * the m_s survivor rows surv_dev[m_s][d] to the new point xn_dev[j] carries the
 * label want_dev[j], else 0 (the sampler then returns the walker's start point).
 * FP32 squared distances accumulated over the coordinates in order by fused
 * multiply-add; ties go to the lower survivor row; m_s = 0 keeps every point.
 * All arrays are caller-owned device memory; m_s, k <= 16384, d <= 512;
 * NS_ERR_ARG otherwise.  Synchronises `stream`. */
ns_status ns_territory(const float *surv_dev, const int *surv_label_dev, int m_s, const float *xn_dev,
                       const int *want_dev, int k, int d, int *keep_dev, void *stream);

/* Order of n log-likelihoods (ascending, NaN first, ties by index):
 * order_dev[n].  n <= 16384. */
ns_status ns_sort_logl(const float *logl_dev, int n, int *order_dev, void *stream);

/* Appendix H statistics for a kill sequence on the device (the same kernel the
 * sampler uses): clusters 0..n_clusters-1 start with counts_host[c] live points,
 * log X = logx0_host[c], log X^2 = 2 log X, log ZX = logzx0_host[c] (may be
 * NULL: -inf), log X_cX_q = logxx0_host[c][q] (may be NULL: -inf); the k kills
 * have labels labels_host[k] (ascending log-likelihood order) and log-likelihoods
 * logl_host[k].  out_host[3 + 3 n_clusters + k] receives log Z, log Z^2, a
 * reserved zero, then per cluster log X, log X^2, log ZX, then the log prior
 * mass of each kill.  NS_ERR_ARG if a cluster loses more points than it has. */
ns_status ns_stats_update(int n_clusters, const int *counts_host, const double *logx0_host,
                          const double *logzx0_host, const double *logxx0_host, int k,
                          const int *labels_host, const double *logl_host, double *out_host);

#ifdef __cplusplus
}
#endif

#endif /* GGNS_H */
