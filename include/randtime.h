/*
 * randtime.h -- C ABI of librandtime: GPU (sm_103a) exact stochastic simulation of
 * chemical reaction networks with the next reaction random time algorithm (NRRTA)
 * of Liu & Wang, "Parallel implementations of random time algorithm for chemical
 * network stochastic simulations", arXiv:2103.00405.
 *
 * Method (the paper's Sec. 2-4):
 *   a_k = c_k h_k(X), h_k = prod_j binom(X_j, sigma_jk)                    Eq. 1-2
 *   X(t) = X(0) + sum_k Y_k(T_k(t)) v_k,  T_k(t) = int_0^t a_k ds           Eq. 16-18
 *   each channel's next firing internal time P_k is a sum of Exp(1)
 *   increments ln(1/r) (Eq. 24); its real waiting time is
 *   dt_k = (P_k - T_k) / a_k (Eq. 25); the smallest fires (Eq. 26); only the
 *   fired channel draws a new increment (Eq. 27, Table 2).
 *
 * Conventions for every entry point:
 *   - Pointers named *_dev are device pointers (cudaMalloc / torch CUDA tensors)
 *     owned by the caller; other pointers are host pointers owned by the caller.
 *     The library owns only the opaque rt_network / rt_batch objects.
 *   - Work is enqueued asynchronously on the CUDA stream `stream` (a cudaStream_t;
 *     NULL = legacy default stream).  Argument errors are detected on the host
 *     before anything is enqueued and returned as a negative rt_status; the message
 *     is available from rt_last_error() (thread-local).
 *   - Per-trajectory outcomes (including numerical overflow) are reported through
 *     the `status` output, never by trapping.
 *   - Counts are int32, times binary64.  All floating-point operations on the
 *     simulation path are single IEEE binary64 operations rounded to nearest, in a
 *     fixed order, so results are bit-identical for a given (network, inputs, seed)
 *     regardless of launch configuration.
 */
#ifndef RANDTIME_H
#define RANDTIME_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Return codes. */
typedef enum {
  RT_OK = 0,
  RT_ERR_INVALID_ARG = -1, /* malformed argument (message in rt_last_error) */
  RT_ERR_UNSUPPORTED = -2, /* valid for the method but not supported here (e.g. order > 2) */
  RT_ERR_CUDA = -3,        /* a CUDA runtime call failed */
  RT_ERR_OOM = -4,         /* device or host allocation failed, or workspace too small */
  RT_ERR_TIMEOUT = -5      /* a bounded device-side wait gave up */
} rt_status;

/* Per-trajectory outcome written to rt_outputs.status. */
enum {
  RT_TRAJ_TEND = 0,       /* the next event would fall after t_end (Table 2 loop condition) */
  RT_TRAJ_MAX_EVENTS = 1, /* max_events events fired */
  RT_TRAJ_ABSORBED = 2,   /* every propensity is zero: no event can ever fire */
  RT_TRAJ_OVERFLOW = 3,   /* the next event would push a count above INT32_MAX (not fired) */
  RT_TRAJ_TIMEOUT = 4,    /* a bounded cross-block wait gave up (bundle and tree mappings) */
  RT_TRAJ_BAD_X0 = 5      /* a negative initial count */
};

/* Trajectory-to-hardware mappings. */
enum {
  RT_MAP_AUTO = -1,  /* chosen by the library from the network size */
  RT_MAP_THREAD = 0, /* one thread per trajectory, state in registers (M <= 16; with M <= 4 and
                        N <= 4 the counts and the network too) */
  RT_MAP_WARP = 1,   /* a warp segment (8, 16 or 32 lanes) per trajectory, channels spread over lanes */
  RT_MAP_BLOCK = 2,  /* one thread block per trajectory, state in registers (M <= 8 * block_threads) */
  RT_MAP_BUNDLE = 3, /* several blocks per trajectory, state streamed through HBM */
  RT_MAP_TREE = 4    /* absolute-time form only: a thread-block cluster per trajectory, min-tree
                        argmin, only the channels an event touches updated */
};

/* Form of the method (rt_run_params.form).  Both simulate the same process with the
 * same random numbers; in exact arithmetic they give the same path, their roundings
 * differ, so each is bit-exact against its own definition. */
enum {
  RT_FORM_INTERNAL = 0, /* Table 2 in internal times: every T_k advanced at every event,
                           T_k += a_k dt, waiting times (P_k - T_k) / a_k for all k */
  RT_FORM_ABSOLUTE = 1, /* absolute firing times with the dependency graph (Sec. 5): channel k
                           keeps s_k (real time of its last update) and
                           tau_k = s_k + (P_k - T_k) / a_k; an event at t = tau_mu touches only
                           mu and the channels reading a changed species:
                           T_k += a_k (t - s_k), s_k = t, P_mu += E, a_k and tau_k recomputed;
                           at the end T_k += a_k (t_f - s_k) with t_f = t_end (run reached it)
                           or the last event time */
  RT_FORM_RESCALED = 2  /* Table 3's form (thread mapping up to M = 8, warp mapping -- a warp per
                           trajectory, a lane per channel -- up to M = 256): relative waiting times w_k;
                           after an event that took dt every propensity is recomputed and every
                           other waiting time rescaled, w_k = (p_k / a_k)(w_k - dt), p_k the
                           previous propensity; the fired channel draws w_mu = E / a_mu; a channel
                           whose propensity is 0 keeps its remaining internal time p_k (w_k - dt)
                           frozen and resumes with w_k = q_k / a_k; T_k += a_k dt per event */
};

typedef struct rt_network rt_network;
typedef struct rt_batch rt_batch;

/* Launch configuration; any field <= 0 (or mapping = RT_MAP_AUTO) means "choose". */
typedef struct rt_launch_cfg {
  int32_t mapping;       /* RT_MAP_* */
  int32_t block_threads; /* threads per block */
  int32_t ctas_per_traj; /* RT_MAP_BUNDLE, RT_MAP_TREE: blocks cooperating on one trajectory */
  int32_t lanes_per_traj; /* RT_MAP_WARP: lanes per trajectory (8, 16 or 32; 32 / lanes
                             trajectories share a warp, at most 8 channels per lane) */
} rt_launch_cfg;

/* What to simulate. */
typedef struct rt_run_params {
  const int32_t *x0_dev;  /* initial counts: [N], or [n_traj][N] if per_traj_x0 */
  int32_t per_traj_x0;
  uint32_t stream_id;     /* 4th Philox counter word: independent streams per network */
  double t_end;           /* simulate on [0, t_end]; +inf allowed when max_events bounds the run */
  int64_t max_events;     /* per-trajectory event cap, 0 <= max_events <= INT32_MAX */
  uint64_t seed;          /* Philox key */
  int64_t n_traj;         /* number of trajectories, >= 0 */
  int64_t traj_offset;    /* global id of trajectory 0 (Philox counter word 1 = lo32(offset + j)) */
  double sample_dt;       /* grid spacing; <= 0: no grid.  Grid times are i*sample_dt, i < G */
  int32_t form;           /* RT_FORM_* (0: internal-time form) */
  int32_t reserved;
} rt_run_params;

/* Where results go.  Any pointer may be NULL (output not produced). */
typedef struct rt_outputs {
  int32_t *x_final_dev;    /* [n_traj][N] state at the end of the run */
  int32_t *grid_dev;       /* [n_traj][G][N] X at grid times (right-continuous); -1 = unknown */
  int64_t *grid_sum_dev;   /* [G][N] += sum over trajectories of X(g) (wraps mod 2^64) */
  int64_t *grid_sumsq_dev; /* [G][N] += sum over trajectories of X(g)^2 */
  int64_t *grid_count_dev; /* [G]    += number of trajectories whose X(g) is known */
  int64_t *n_events_dev;   /* [n_traj] events fired */
  int32_t *status_dev;     /* [n_traj] RT_TRAJ_* */
  double *t_last_dev;      /* [n_traj] time of the last fired event (0 if none) */
  double *loglik_dev;      /* [n_traj] path log-likelihood sum ln a_mu - sum_k T_k(t_end) */
  int32_t *counts_dev;     /* [n_traj][M] firings n_k per channel */
  double *t_internal_dev;  /* [n_traj][M] internal times T_k(t_end) */
  int64_t trace_len;       /* events recorded per trajectory in trace_*_dev (0: no trace) */
  int32_t *trace_mu_dev;   /* [n_traj][trace_len] channel fired by event e (Table 2's triggered j);
                              -1 after the trajectory's last event */
  double *trace_t_dev;     /* [n_traj][trace_len] time t of event e (after the update t += dt);
                              0 after the trajectory's last event */
} rt_outputs;

/*
 * rt_network_create -- validate and pack a network, copying it to the current device.
 *
 * Network in COO form as the paper stores it (Sec. 5, "Implementations"):
 *   reactant coefficients sigma (reac_*: n_reac_nz entries, coef > 0) and net
 *   state change v (stoi_*: n_stoi_nz entries), rates c[n_reactions] (Eq. 1).
 * All arrays are host arrays, read during the call only.  Duplicate (reaction,
 * species) entries are summed.  Requirements (else RT_ERR_INVALID_ARG):
 * 1 <= n_species, 1 <= n_reactions, indices in range, c finite and >= 0, and a
 * negative net change only on a reactant species with |v| <= sigma (counts can
 * never go negative).  A reaction with more than two reactant molecules returns
 * RT_ERR_UNSUPPORTED (the paper's two-reactant limit, Sec. 5).
 * On success *out owns device memory until rt_network_destroy.
 */
int rt_network_create(int32_t n_species, int32_t n_reactions,
                      int64_t n_reac_nz, const int32_t *reac_rxn, const int32_t *reac_sp,
                      const int32_t *reac_coef,
                      int64_t n_stoi_nz, const int32_t *stoi_rxn, const int32_t *stoi_sp,
                      const int32_t *stoi_delta,
                      const double *c, rt_network **out);

/* Free a network (NULL is ignored).  The caller must ensure no work using it is in flight. */
void rt_network_destroy(rt_network *net);

/*
 * rt_network_info -- sizes of a packed network.  Any output pointer may be NULL.
 * max_dependents: the largest number of channels whose propensity one firing can
 * change (the Gibson-Bruck dependency graph the paper mentions in Sec. 5).
 */
int rt_network_info(const rt_network *net, int32_t *n_species, int32_t *n_reactions,
                    int32_t *max_dependents, int64_t *n_dependency_nz);

/*
 * rt_network_set_enabled -- forbid channels to fire (the paper's boundary conditions:
 * a forbidden channel is given a frozen internal time, Table 2's note).  enabled: host
 * array [n_reactions], 0 = forbidden (its propensity is taken as 0, so its internal
 * time stays frozen and it never fires); NULL enables every channel.  The network's
 * own rates are kept: rt_loglik_backward still divides by them, so a forbidden
 * channel's gradient is 0.  Copies to the device synchronously; no work using the
 * network may be in flight.  Batches created afterwards take the setting with them.
 */
int rt_network_set_enabled(rt_network *net, const uint8_t *enabled);

/*
 * rt_network_set_rate_slopes -- time-dependent rates c_k(t) = c_k (1 + beta_k t) (Sec. 6,
 * Eq. 29: in the random-time form each channel needs only its own integral, here in closed
 * form).  beta: host array [n_reactions], finite and >= 0; NULL returns to constant rates.
 * Between events channel k's internal time grows by A_k I_k(t, dt), A_k = c_k h_k(X),
 * I_k = dt (1 + beta_k t) + beta_k dt^2 / 2; its waiting time is the root of
 * A_k I_k(t, dt) = P_k - T_k, dt = 2R / (b + sqrt(b^2 + 2 A_k beta_k R)) with
 * u = 1 + beta_k t, b = A_k u, R = P_k - T_k (for beta_k = 0: R / A_k, the constant-rate
 * operations); ln a_mu is taken at the event time.  The gradient (n_k - T_k) / c_k keeps
 * its form.  Networks with slopes run the internal-time form on the thread mapping
 * (M <= 16) or the warp mapping (M <= 256, 32 lanes per trajectory; the default above
 * 16 reactions); other mappings, forms and batches return RT_ERR_UNSUPPORTED.  Copies to
 * the device synchronously; no work using the network may be in flight.
 */
int rt_network_set_rate_slopes(rt_network *net, const double *beta);

/* Number of grid points on [0, t_end] for spacing sample_dt:
 * floor(t_end / sample_dt * (1 + 1e-12)) + 1, or 0 if sample_dt <= 0 or t_end is not finite. */
int64_t rt_grid_len(double t_end, double sample_dt);

/*
 * rt_workspace_bytes -- device scratch that rt_run needs for this network, run and
 * launch configuration (0 for register/shared-memory mappings).  The caller
 * allocates it (>= 256-byte aligned) and passes it to rt_run.
 */
int rt_workspace_bytes(const rt_network *net, const rt_run_params *params, const rt_launch_cfg *cfg,
                       size_t *bytes);

/*
 * rt_run -- simulate params->n_traj independent trajectories of `net` (Table 2 of
 * the paper in internal-time form: Eq. 24-27).
 *
 * Per trajectory j (global id g = traj_offset + j): X = X0, t = 0, T_k = 0,
 * P_k = E(g,k,0), a_k = c_k h_k(X); then repeatedly: dt_k = (P_k - T_k)/a_k
 * (+inf if a_k = 0, 0 if P_k <= T_k), mu = argmin (smallest k on ties); stop if
 * no channel can fire, if t + dt_mu > t_end, if max_events fired, or if firing
 * would overflow int32; else t += dt_mu, T_k += a_k dt_mu for all k, X += v_mu,
 * P_mu += E(g, mu, n_mu), recompute a_k for the channels that depend on the
 * changed species.  E(g,k,n) is the Philox4x32-10 Exp(1) draw described in
 * rt_draw_exp1.  Grid samples use X after all events at times <= the grid time.
 * With loglik/counts/t_internal outputs, T_k is advanced to t_end at the end
 * (when the run reached t_end or was absorbed) and the log-likelihood
 * sum_events ln a_mu - sum_k T_k (summed in k order) is written.
 *
 * params->form selects the form of the method (RT_FORM_*): the absolute-time form
 * runs on RT_MAP_TREE only, Table 3's form on the thread (M <= 8) or warp (M <= 256)
 * mapping; a network with rate slopes (rt_network_set_rate_slopes) runs the
 * internal-time form on the thread (M <= 16) or warp (M <= 256) mapping; forbidden
 * channels (rt_network_set_enabled) are honoured by every mapping and form.  Other
 * combinations return RT_ERR_UNSUPPORTED before anything is enqueued.
 *
 * x0 values are checked on the device (negative -> RT_TRAJ_BAD_X0).  workspace
 * must be at least rt_workspace_bytes() (may be NULL when that is 0).
 * grid_sum/sumsq/count are accumulated into (+=): zero them first.
 */
int rt_run(const rt_network *net, const rt_run_params *params, const rt_outputs *outputs,
           const rt_launch_cfg *cfg, void *workspace_dev, size_t workspace_bytes, void *stream);

/*
 * rt_run_bundle_noalloc -- rt_run with the bundle mapping (RT_MAP_BUNDLE) that
 * allocates nothing and needs no workspace from the caller.  The paper has no
 * counterpart; it exists for callers that cannot call cudaMalloc where they run a
 * simulation, such as a host application whose device memory is owned by its own
 * pool allocator, or a latency-critical loop that must stay out of the driver's
 * allocator (which can synchronise the device).
 *
 * Arguments and results are those of rt_run with cfg->mapping = RT_MAP_BUNDLE and
 * cfg->ctas_per_traj = ctas_per_traj (<= 0: chosen by the library).  The scratch
 * lives in a fixed 16 MiB device array inside the library, which every GPU that
 * loads the library holds until the process exits; a run that needs more (about
 * 28 bytes per channel per trajectory plus a few KB) returns RT_ERR_OOM with a
 * message, and nothing is enqueued.  Every call looks up that array's device
 * address on the current device (cudaGetSymbolAddress, which allocates nothing), so
 * a device reset between calls is harmless; the first call on a device loads the
 * library's device code there, so make it before any stream capture.  All calls on
 * a device share the array
 * and it keeps the last call's contents: calls whose work overlaps on the GPU
 * (different streams, or threads without ordering) race on it, so order them on
 * one stream or synchronise between them.
 */
int rt_run_bundle_noalloc(const rt_network *net, const rt_run_params *params, const rt_outputs *outputs,
                          int32_t ctas_per_traj, void *stream);

/*
 * rt_loglik_backward -- gradient of sum_j grad_ll[j] * l_j with respect to the
 * rate constants, from the counts and internal times saved by rt_run:
 *   grad_c[k] = sum_j grad_ll[j] * (n_jk - T_jk(t_end)) / c_k
 * (d l / d c_k = n_k / c_k - int h_k dt, since T_k = c_k int h_k dt; Eq. 16-18).
 * grad_ll_dev [n_traj], counts_dev [n_traj][M], t_internal_dev [n_traj][M],
 * grad_c_dev [M] (overwritten).  Entries with c_k = 0 come out as NaN.
 */
int rt_loglik_backward(const rt_network *net, int64_t n_traj, const double *grad_ll_dev,
                       const int32_t *counts_dev, const double *t_internal_dev, double *grad_c_dev,
                       void *stream);

/*
 * rt_draw_exp1 -- the Exp(1) internal-time increments of Eq. 24, E = ln(1/u), for
 * count (traj, channel, index) triples (device arrays), as used by rt_run.
 * Philox4x32-10 (Salmon et al., SC'11) with key (lo32(seed), hi32(seed)) and
 * counter (index >> 1, lo32(traj), channel, stream_id); an even index takes
 * output words (w0, w1), an odd one (w2, w3); v = (w1:w0) >> 12 and
 * u = (2v + 1) 2^-53.  ln is a fixed-point evaluation (error <= 0.51 ulp)
 * rounded once to binary64.  Writes u to u_dev and E to e_dev (either may be NULL).
 */
int rt_draw_exp1(uint64_t seed, uint32_t stream_id, int64_t count, const uint64_t *traj_dev,
                 const uint32_t *channel_dev, const uint64_t *index_dev, double *u_dev, double *e_dev,
                 void *stream);

/* rt_log_eval -- the library's natural logarithm (used for ln a_mu) of count positive
 * finite doubles x_dev, into y_dev. */
int rt_log_eval(int64_t count, const double *x_dev, double *y_dev, void *stream);

/* rt_philox -- raw Philox4x32-10 blocks: out_dev[4i..4i+3] = philox(ctr_dev[4i..], key). */
int rt_philox(int64_t count, const uint32_t *ctr_dev, uint32_t key0, uint32_t key1, uint32_t *out_dev,
              void *stream);

/*
 * Batched mode: many networks of uneven size in one persistent launch.
 *
 * The paper groups the blocks of one trajectory into a "bundle" (Sec. 5); here
 * thousands of independent networks share one launch.  Each network is assigned
 * a mapping class by size: one thread per trajectory (M <= thread_max_m), one
 * warp (M <= warp_max_m), or one block of block_threads threads (M <= 16 *
 * block_threads).  Work is a list of block-sized tasks (one block-class
 * trajectory, block_threads/32 warp-class or block_threads thread-class
 * trajectories), larger networks first, that persistent blocks take from an
 * atomic counter.  Network i draws its random numbers with its own stream id
 * (default i), so its trajectories equal rt_run of that network with that stream id.
 */
typedef struct rt_batch_policy {
  int32_t thread_max_m;  /* <= 8; networks with more than 8 species go to the warp class */
  int32_t warp_max_m;    /* <= 256 */
  int32_t block_threads; /* threads per block: 128, 256 or 512 */
  int32_t blocks_per_sm; /* persistent blocks per SM; 0 = as many as fit */
} rt_batch_policy;

/* Pack the networks into one device arena (the batch keeps its own copy; the
 * network handles may be destroyed afterwards).  stream_ids: host array [n_nets],
 * the Philox stream (fourth counter word) of each network's draws, or NULL for
 * network i -> stream i; a run sharded over several GPUs passes each network's
 * global index so its trajectories equal the single-GPU run's.  policy may be NULL
 * (defaults 8 / 256 / 512 / 0).  All networks must live on the current device.
 * Networks too large for the block class (M > 16 * block_threads) return
 * RT_ERR_UNSUPPORTED. */
int rt_batch_create(int32_t n_nets, const rt_network *const *nets, const uint32_t *stream_ids,
                    const rt_batch_policy *policy, rt_batch **out);
void rt_batch_destroy(rt_batch *batch);

/* Totals of the packed batch: species (length of packed x0), reactions, and the
 * number of networks in each class (thread, warp, block).  Any pointer may be NULL. */
int rt_batch_info(const rt_batch *batch, int64_t *total_species, int64_t *total_reactions, int32_t *n_thread_class,
                  int32_t *n_warp_class, int32_t *n_block_class);

/* Where a batched run's results go.  Any pointer may be NULL (output not produced).
 * Network i has N_i species and M_i reactions; "packed" arrays hold network after
 * network, each as [traj j][N_i] or [traj j][M_i] (the offsets are n_traj times the
 * sums of N or M over the networks before i). */
typedef struct rt_batch_outputs {
  int32_t *x_final_dev;    /* packed [net i][traj j][N_i] final states */
  int64_t *n_events_dev;   /* [n_nets][n_traj] events fired */
  int32_t *status_dev;     /* [n_nets][n_traj] RT_TRAJ_* */
  double *t_last_dev;      /* [n_nets][n_traj] time of the last fired event */
  double *loglik_dev;      /* [n_nets][n_traj] path log-likelihood, as rt_outputs.loglik_dev */
  int32_t *counts_dev;     /* packed [net i][traj j][M_i] firings n_k */
  double *t_internal_dev;  /* packed [net i][traj j][M_i] internal times T_k(t_end) */
  int64_t trace_len;       /* events recorded per trajectory (0: none) */
  int32_t *trace_mu_dev;   /* [n_nets][n_traj][trace_len] fired channels, -1 after the last event */
  double *trace_t_dev;     /* [n_nets][n_traj][trace_len] event times, 0 after the last event */
} rt_batch_outputs;

/*
 * rt_batch_run -- n_traj_per_net trajectories of every network, in one launch
 * (plus a counter reset), enqueued on `stream` without host synchronisation, so
 * it can be captured in a CUDA graph.
 *   x0_dev:    initial counts, network after network (sum of N_i int32)
 *   t_end_dev: [n_nets] horizons (finite, >= 0)
 *   outputs:   rt_batch_outputs (NULL: nothing written)
 * max_events caps every trajectory (0 <= max_events <= INT32_MAX).  Network i's
 * trajectory j equals rt_run of that network with stream_id = its stream id and
 * traj_offset = 0 (trajectory j), bit for bit.
 */
int rt_batch_run(rt_batch *batch, const int32_t *x0_dev, const double *t_end_dev, int64_t max_events,
                 uint64_t seed, int64_t n_traj_per_net, const rt_batch_outputs *outputs, void *stream);

/*
 * rt_fp64_probe -- a measurement aid with no counterpart in the paper: launches
 * blocks_per_sm x (number of SMs) blocks of 256 threads, each thread running 8
 * independent chains of `iters` binary64 multiply-then-add steps (never fused),
 * so that the time of the launch (taken by the caller with CUDA events on
 * `stream`) gives the GPU's binary64 add/multiply issue rate.  *ops (host
 * pointer, may be NULL) receives the number of binary64 operations the launch
 * performs.  sink_dev: one device double, written only in a case that never
 * happens (it keeps the loop from being optimised away).
 */
int rt_fp64_probe(int64_t iters, int32_t blocks_per_sm, double *sink_dev, double *ops, void *stream);

/*
 * Model files (the text format of the paper's Table 4, Sec. 5):
 *   // comment
 *   # init
 *   A = 1000                      initial counts
 *   # reactions
 *   1 A 1 B --> 2 B : 0.01        coef name ... --> coef name ... : rate (NULL: none;
 *                                 a coefficient 1 may be omitted; "->" also accepted)
 *   # end
 *   time = 2                      settings after "# end"
 *   steps = 10000
 * Species are numbered in order of first appearance; species that appear only in
 * reactions start at 0.  The network comes out in the COO form of rt_network_create.
 */
typedef struct rt_model {
  int32_t n_species, n_reactions;
  int64_t n_reac_nz;
  int32_t *reac_rxn, *reac_sp, *reac_coef;  /* reactant coefficients (merged per species) */
  int64_t n_stoi_nz;
  int32_t *stoi_rxn, *stoi_sp, *stoi_delta; /* net state changes (nonzero only) */
  double *c;                                /* [n_reactions] rates */
  int32_t *x0;                              /* [n_species] initial counts */
  char **species_names;                     /* [n_species] NUL-terminated names */
  double time;                              /* "time" setting, NaN if absent */
  int64_t steps;                            /* "steps" setting, -1 if absent */
} rt_model;

/* Parse model text (host, NUL-terminated).  On success *out is owned by the library until
 * rt_model_free.  Malformed text returns RT_ERR_INVALID_ARG with the line in rt_last_error. */
int rt_model_parse(const char *text, rt_model **out);
void rt_model_free(rt_model *model);

/* Message describing the last error on this host thread ("" if none). */
const char *rt_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* RANDTIME_H */
