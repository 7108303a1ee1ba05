/*
 * smc.h -- C ABI of the GB300 statistical model checking library.
 *
 * The library estimates P(phi) for a mass-action reaction network and a
 * time-bounded BLTLc formula phi, as in Ballarini, Forlin, Mazza and Prandi,
 * "Efficient Parallel Statistical Model Checking of Biochemical Networks"
 * (PDMC 2009): it generates independent trajectories with Gillespie's direct
 * method (Sec. 2.2, Eq. 1, 2a, 2b), checks each one on the fly against phi
 * (Sec. 3.1 semantics, Sec. 3.2 on-the-fly verification) and stops it as soon
 * as its verdict is fixed, and reduces the verdicts into the Wilson score
 * interval (Eq. 4) with the iterative sample-size rule (Eq. 5, Fig. 2).
 *
 * Every step of that path runs in the library's own CUDA kernels on one GPU.
 *
 * Conventions for every entry point:
 *  - Return value: SMC_OK (0) or a negative SMC_E_* code; no exceptions
 *    cross the ABI.  smc_last_error() gives a message for the last failure
 *    on a context.
 *  - Host pointers are read during the call only; the library copies what
 *    it keeps (the caller keeps ownership).  Pointers documented as device
 *    pointers must be device memory of the context's GPU (for example from
 *    torch), owned by the caller.
 *  - A context is used by one host thread at a time; calls on one context do
 *    not overlap.  Work is issued on the context's stream unless a stream is
 *    passed; entry points that return host results synchronise with it.
 *  - Trajectory indices are 32-bit per instance (fewer than 2^32
 *    trajectories per instance per seed).
 */
#ifndef SMC_H
#define SMC_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- return codes ------------------------------------------------------ */
#define SMC_OK 0
#define SMC_E_INVALID_ARG (-1) /* bad shape, negative or non-finite rate, ... */
#define SMC_E_OOM (-2)         /* device or host allocation failed             */
#define SMC_E_CUDA (-3)        /* a CUDA call failed; see smc_last_error       */
#define SMC_E_UNSUPPORTED (-4) /* formula outside the monitorable fragment     */
#define SMC_E_STATE (-5)       /* call order: no model / property loaded       */
#define SMC_E_NO_DEVICE (-6)   /* no CUDA device, or not a device of sm_103    */

/* ---- per-instance status bits (smc_result.status) ----------------------- */
#define SMC_STATUS_BUDGET 1 /* some trajectories exhausted the event budget */

/* ---- arithmetic of the SSA path ----------------------------------------- */
#define SMC_PLAIN_FP64 0 /* FP64 propensities, selection and clock          */
#define SMC_MIXED 1      /* FP32 propensities and selection, exact int32
                            counts, FP64 clock, FP64 renormalisation of a_0
                            every 2^k events                                */

/* ---- sample size rule (smc_estimate mode, bits 4..7) --------------------- */
#define SMC_FIXED_N (0 << 4)      /* run exactly fixed_n trajectories           */
#define SMC_ITERATIVE (1 << 4)    /* Fig. 2, starting from p = 1                */
#define SMC_CONSERVATIVE (2 << 4) /* one batch of Wilson_sample(0.5) (Sec. 3.3.1) */

/* ---- formula nodes (postfix order) -------------------------------------- */
#define SMC_NODE_TRUE 0
#define SMC_NODE_FALSE 1
#define SMC_NODE_ATOM 2       /* arg = atom index                          */
#define SMC_NODE_NOT 3        /* 1 operand                                 */
#define SMC_NODE_AND 4        /* 2 operands                                */
#define SMC_NODE_OR 5         /* 2 operands                                */
#define SMC_NODE_IMPLIES 6    /* 2 operands                                */
#define SMC_NODE_UNTIL 7      /* phi U[lo,hi] psi: 2 operands (phi first)  */
#define SMC_NODE_EVENTUALLY 8 /* F[lo,hi] psi = tt U[lo,hi] psi            */
#define SMC_NODE_ALWAYS 9     /* G[lo,hi] psi = not F[lo,hi] not psi       */
#define SMC_NODE_NEXT 10      /* X[lo,hi] psi: the next state is entered at
                                 a time in [lo, hi] and satisfies psi (Sec.
                                 3.1)                                       */

/* ---- atom comparison operators ------------------------------------------ */
#define SMC_OP_LT 0
#define SMC_OP_LE 1
#define SMC_OP_GE 2
#define SMC_OP_GT 3
#define SMC_OP_EQ 4
#define SMC_OP_NE 5

/* ---- options (smc_set_option) ------------------------------------------- */
#define SMC_OPT_EVENT_BUDGET 0    /* max reactions per trajectory (default 2^24) */
#define SMC_OPT_RENORM_LOG2 1     /* mixed path: a_0 renormalised every 2^k events (default 8) */
#define SMC_OPT_AUTOTUNE 2        /* 1 = choose launch shape by timed trials (default 1);
                                     the result is kept for later loads of a model of
                                     the same structure (instances, S, R per size class) */
#define SMC_OPT_WARPS_PER_BLOCK 3 /* fixed launch shape when autotune is 0 (default 4) */
#define SMC_OPT_BLOCKS_PER_SM 4   /* 0 = as many as fit (default 0) */
#define SMC_OPT_REFILL 5          /* refill a warp when >= this many lanes idle (default 1) */
#define SMC_OPT_RECORD 6          /* 1 = keep per-trajectory verdicts of FIXED_N estimates */
#define SMC_OPT_JIT 7             /* 1 = model-specialized kernels when every instance shares one
                                     structure with S, R <= 32 (default 1; compiled at run time
                                     with NVRTC, same results as the generic kernels) */
#define SMC_OPT_SELECTION 8       /* reaction selection of the generic kernel (Eq. 2b):
                                     0 = automatic (running sums checkpointed every 16
                                     reactions for networks of more than 64 reactions,
                                     else a linear scan), 1 = linear scan, 2 = checkpoints
                                     for networks of more than 16 reactions; the same
                                     trajectories in every mode (default 0) */
#define SMC_OPT_TRACE_CAP 9       /* trace monitor (formulas nested beyond the monitor's
                                     units, see smc_load_property): positions each lane
                                     records per trajectory, 16..2^24 (default 4096); a
                                     trajectory that needs more gets status 3.  Device
                                     memory: lanes x cap x (12 + 4 x memo slots) bytes,
                                     one memo slot per temporal operator nested inside
                                     another (116,736 lanes, the FP64 path's default
                                     shape on a GB300: 1.4 GB per 1024 positions, plus
                                     0.5 GB per slot); SMC_E_OOM when it does not fit */

/* A node of the formula in postfix order: operands precede their operator. */
typedef struct {
    int32_t kind; /* SMC_NODE_*                                            */
    int32_t arg;  /* atom index for SMC_NODE_ATOM, else ignored            */
    double lo;    /* interval [lo, hi] of UNTIL / EVENTUALLY / ALWAYS,      */
    double hi;    /* 0 <= lo <= hi; hi may be +inf (unbounded, see t_max)   */
} smc_node;

/* Per-instance estimate. */
typedef struct {
    double p_hat;         /* yes / n                                          */
    double lo, hi;        /* Wilson score interval, Eq. 4                      */
    uint64_t n;           /* trajectories with a verdict                       */
    uint64_t yes;         /* trajectories that satisfy phi                     */
    uint64_t launched;    /* trajectories simulated = n + budget_hits          */
    uint64_t events;      /* reactions fired, summed over trajectories         */
    uint64_t budget_hits; /* trajectories stopped by the event budget          */
    int32_t status;       /* SMC_STATUS_* bits                                 */
    int32_t iterations;   /* Fig. 2 iterations performed                       */
} smc_result;

/* Device-side outputs of smc_simulate (all device pointers; NULL = skip). */
typedef struct {
    uint64_t *counts; /* [n_inst][4]: yes, n, events, budget_hits; ADDED to  */
    double *wilson;   /* [n_inst][3]: p_hat, lo, hi of the counts after the call */
    uint8_t *verdict; /* [n_inst][n_traj]: 1 = phi holds                      */
    uint8_t *status;  /* [n_inst][n_traj]: 0 decided, 1 event budget, 3 the
                         trace monitor's recording full (or undecided past
                         4 t_horizon + 1); 1 and 3 count as budget_hits      */
    uint64_t *events; /* [n_inst][n_traj]: reactions fired                    */
    double *t_final;  /* [n_inst][n_traj]: entry time of the last state       */
    int32_t *x_final; /* [n_inst][n_traj][S_max]: last state                  */
} smc_sim_out;

typedef struct smc_ctx smc_ctx;

/* Creates a context on CUDA device `device`.  *out receives the handle.
 * Errors: SMC_E_NO_DEVICE (no such device / not compute capability 10.3),
 * SMC_E_OOM, SMC_E_CUDA. */
int smc_create(smc_ctx **out, int device);

/* Releases the context and its device memory.  NULL is ignored. */
void smc_destroy(smc_ctx *ctx);

/* Static description of an error code. */
const char *smc_strerror(int code);

/* Message of the last failure on ctx ("" if none). */
const char *smc_last_error(const smc_ctx *ctx);

/* Loads one reaction network (Sec. 2.2) with n_instances parameter sets.
 *  reactants [R][2]: species index of each reactant or -1 (reaction order
 *      <= 2; two equal indices = homodimer S_a + S_a, propensity
 *      c x_a (x_a - 1) / 2; one index: c x_a; none: c; two: c x_a x_b).
 *  stoich [R][S]: net change v_ji of species i when reaction j fires.
 *  rates [n_instances][R]: stochastic rate constants c_j (finite, >= 0).
 *  x0 [n_instances][S]: initial counts (>= 0).
 * Replaces any previous model.  Errors: SMC_E_INVALID_ARG. */
int smc_load_model(smc_ctx *ctx, int n_species, int n_reactions, const int32_t *reactants,
                   const int32_t *stoich, const double *rates, const int32_t *x0,
                   int n_instances);

/* Loads n_instances networks of different sizes in one batch.
 *  n_species[m], n_reactions[m]: sizes of instance m (1..255 each).
 *  reactants, stoich, rates, x0: the per-instance arrays of
 *  smc_load_model concatenated in instance order ([R_m][2], [R_m][S_m],
 *  [R_m], [S_m]). */
int smc_load_model_batch(smc_ctx *ctx, int n_instances, const int32_t *n_species,
                         const int32_t *n_reactions, const int32_t *reactants,
                         const int32_t *stoich, const double *rates, const int32_t *x0);

/* Loads the property (Sec. 3.1): atoms  sum_i coef[a][i] x_i  <op[a]>  bound[a]
 * with integer coefficients, and a formula over them in postfix order.
 *  atom_coef [n_atoms][S] (single network) -- or, after
 *      smc_load_model_batch, [n_inst] blocks of [n_atoms][S_m];
 *  atom_op [n_atoms]: SMC_OP_*;  atom_bound [n_atoms] (or [n_inst][n_atoms]
 *      when per_instance != 0): finite bounds;
 *  t_max_unbounded: horizon of the pessimistic rule (Sec. 3.2) for
 *      formulas with an infinite interval end: a trajectory still undecided
 *      when its clock passes t_max is counted false.
 * The library compiles the formula into a monitor automaton when it can:
 * boolean combinations (<= 4 temporal operators, <= 6 distinct atoms) of
 * U[a,b], F[a,b], G[a,b] whose left operand is a state formula and whose
 * right operand is a state formula, or a state formula AND F[0,d] / G[0,d]
 * of a state formula (after pushing negations inward), and X[a,b] of a
 * state formula at the top level.  Any other formula of the grammar (Sec.
 * 3.1: U, F, G, X nested in either operand, to a tree height of 10 and 32
 * nodes, <= 6 distinct atoms) runs on the trace monitor: each lane records
 * its trajectory (entry times, atoms; SMC_OPT_TRACE_CAP positions) and the
 * formula's verdict, and the first point at which it is fixed, are computed
 * from the recording (Sec. 3.2's lookahead buffer) on a doubling schedule of
 * events and at the formula's horizon; the trajectory then reports the
 * events, clock and state of that point, as if it had stopped there.  The
 * trace monitor runs on the generic kernels only, and not under
 * smc_simulate_noalloc, smc_simulate_snapshot or smc_estimate_cv (those
 * return SMC_E_UNSUPPORTED).  Beyond its limits: SMC_E_UNSUPPORTED. */
int smc_load_property(smc_ctx *ctx, int n_atoms, const int32_t *atom_coef,
                      const int32_t *atom_op, const double *atom_bound, int per_instance,
                      const smc_node *nodes, int n_nodes, double t_max_unbounded);

/* Which monitor the loaded property runs on: 1 the monitor's units, 2 the
 * trace monitor (see smc_load_property), 0 no property loaded (or ctx NULL). */
int smc_monitor_kind(const smc_ctx *ctx);

/* Rate-law factors beyond mass action.  Sec. 2.2 uses mass-action
 * propensities; the cell-cycle model of Sec. 5 needs rational rate laws
 * (Michaelis-Menten and Hill terms, J + alpha y denominators).  Factor q
 * multiplies the propensity of reaction reaction[q] by
 *     (a0 + a1 x^n) / (b0 + b1 x^n),   x = count of species species[q],
 * n = power[q] in 1..4, (a0, a1, b0, b1) = params[4q .. 4q+3], finite, with
 * a0, a1, b1 >= 0 and b0 > 0 (so the factor is finite and >= 0), at most 2
 * factors per reaction, applied in the order given:
 *     a = c h (mass action);  per factor: xn = x, then xn *= x (n - 1
 *     times); num = a0 + a1 xn; den = b0 + b1 xn; a = a * (num / den),
 * every operation rounded once (FP64 on the FP64 path, FP32 on the mixed
 * path).  A factor with a0 = 0 vanishes with its species, which lets a
 * reaction consume a species it does not take as a mass-action reactant
 * (e.g. Michaelis-Menten degradation: zeroth-order mass action, stoichiometry
 * -1, factor x / (K + x)); keeping counts non-negative is the model's
 * responsibility, as for mass action.  Applies to every instance of the model
 * loaded with smc_load_model (host arrays, copied); a later smc_load_model
 * clears the factors; n_factors = 0 removes them.  Errors: SMC_E_STATE before
 * a model is loaded, SMC_E_UNSUPPORTED after smc_load_model_batch,
 * SMC_E_INVALID_ARG for an index, power, parameter or count out of range. */
int smc_load_rate_factors(smc_ctx *ctx, int n_factors, const int32_t *reaction, const int32_t *species,
                          const int32_t *power, const double *params);

/* Exact time-bounded reachability for the loaded property on one instance,
 * by uniformisation of the CTMC (Sec. 2.2's chain solved numerically): the
 * exact side of the comparison of Sec. 5 / Fig. 4 (there done with PRISM),
 * as a validator of smc_estimate.  No counterpart in the paper's own method.
 * The property must compile to one L U[0,b] P, F[0,b] P or G[0,b] P over
 * state formulas (b finite).  The states reachable from x0 are enumerated on
 * the host (at most max_states; states with a count above cap are absorbing
 * and their mass by b is reported as `truncated`, which bounds the error
 * from above); the uniformised chain's iterations run on the GPU in FP64.
 * Synchronous.  Errors: SMC_E_STATE (no model or property), SMC_E_UNSUPPORTED
 * (formula shape, or more reachable states than max_states),
 * SMC_E_INVALID_ARG (instance, cap, a count driven negative), SMC_E_CUDA,
 * SMC_E_OOM. */
typedef struct {
    double p;            /* P(phi) up to the truncation below            */
    double truncated;    /* probability mass in capped states by b       */
    double poisson_tail; /* Poisson weight left out (about 1e-14)        */
    int64_t n_states;    /* reachable states enumerated                  */
    int64_t iterations;  /* uniformisation steps                         */
    double lambda_t;     /* uniformisation rate x b                      */
} smc_cme_result;
int smc_cme_reach(smc_ctx *ctx, int instance, int32_t cap, int64_t max_states, smc_cme_result *out);

/* Arithmetic atoms (Sec. 3.1's grammar: val <| val with val built from
 * counts, constants, + - * / and functions such as sqrt and pow).  Atom
 * `atom` of the loaded property becomes  lhs <op> rhs,  each side a postfix
 * program of tokens evaluated in FP64, every operation rounded once
 * (IEEE: x / 0 is +-inf, sqrt of a negative is NaN, and every comparison
 * with NaN is false except !=):
 *   SMC_TOK_SPECIES  push (double) x[arg]      SMC_TOK_CONST  push value
 *   SMC_TOK_ADD / SUB / MUL / DIV  pop b, pop a, push a <op> b
 *   SMC_TOK_SQRT     pop a, push sqrt(a) (correctly rounded)
 *   SMC_TOK_POWI     pop a, push a^arg, arg in 0..16, by repeated
 *                    multiplication left to right (a^0 = 1)
 * A program must leave exactly one value, with a stack of at most
 * SMC_EXPR_MAX_DEPTH and at most SMC_EXPR_MAX_TOKENS tokens per side.  The
 * atom's coefficients and bound given to smc_load_property are then
 * ignored; the expression applies to every instance (batched networks: to
 * species indices valid in every instance).  Call after smc_load_property
 * (which clears expressions).  Errors: SMC_E_STATE before a property is
 * loaded, SMC_E_INVALID_ARG for a bad atom index, operator, token, species or
 * program shape. */
#define SMC_TOK_SPECIES 0
#define SMC_TOK_CONST 1
#define SMC_TOK_ADD 2
#define SMC_TOK_SUB 3
#define SMC_TOK_MUL 4
#define SMC_TOK_DIV 5
#define SMC_TOK_SQRT 6
#define SMC_TOK_POWI 7
#define SMC_EXPR_MAX_DEPTH 8
#define SMC_EXPR_MAX_TOKENS 32
typedef struct {
    int32_t kind;  /* SMC_TOK_*                                   */
    int32_t arg;   /* species index (SPECIES) or exponent (POWI)  */
    double value;  /* constant (CONST)                            */
} smc_token;
int smc_set_atom_expression(smc_ctx *ctx, int atom, int op, const smc_token *lhs, int n_lhs,
                            const smc_token *rhs, int n_rhs);

/* Sets an SMC_OPT_* option.  Errors: SMC_E_INVALID_ARG. */
int smc_set_option(smc_ctx *ctx, int option, double value);

/* Launch shape in use for `precision` (no counterpart in the paper: the
 * batching of Sec. 4's replicas into persistent launches is this library's).
 * The instances are served by *n_launches launches (one per size class, or
 * one over all instances, as the autotuner chose); launch `index` uses
 * *warps_per_block warps per block, *blocks_per_sm resident blocks per SM,
 * refill threshold *refill, serves *n_instances instances, and runs the
 * model-specialized kernel (*specialized = 1, see SMC_OPT_JIT) or the
 * generic one (0).  Any output pointer may be null.  Valid after an estimate
 * or simulation of the loaded model.  Errors: SMC_E_STATE before that,
 * SMC_E_INVALID_ARG for a bad precision or index (*n_launches is still
 * written). */
int smc_get_launch_shape(smc_ctx *ctx, int precision, int index, int *n_launches, int *warps_per_block,
                         int *blocks_per_sm, int *refill, int *n_instances, int *specialized);

/* Estimates P(phi) for every instance (Sec. 3.3).
 *  confidence = 1 - alpha (0 < confidence < 1);
 *  half_width = epsilon of Eq. 5 (> 0; unused for SMC_FIXED_N);
 *  seed keys the counter-based random numbers;
 *  mode = SMC_PLAIN_FP64 or SMC_MIXED, plus SMC_FIXED_N, SMC_ITERATIVE or
 *      SMC_CONSERVATIVE;
 *  fixed_n: trajectories per instance for SMC_FIXED_N;
 *  out [n_instances]: host array receiving the results.
 * Trajectory k of instance m always draws the same random numbers for a
 * given seed, whatever the launch shape, so results are reproducible. */
int smc_estimate(smc_ctx *ctx, double confidence, double half_width, uint64_t seed, int mode,
                 uint64_t fixed_n, smc_result *out);

/* Copies the per-trajectory verdicts ([n_inst][fixed_n], uint8) of the last
 * SMC_FIXED_N smc_estimate run with SMC_OPT_RECORD = 1 into host memory.
 * n must equal n_inst * fixed_n.  Errors: SMC_E_STATE (nothing recorded). */
int smc_get_verdicts(smc_ctx *ctx, uint8_t *out, uint64_t n);

/* Runs trajectories traj_begin .. traj_begin + n_traj - 1 of every
 * instance on `stream` (a cudaStream_t; NULL = the context's stream) and
 * writes the device outputs in *out (counts are added to, so ranges can be
 * chained; wilson is computed with z for `confidence` from the counts after
 * this call).  Does not synchronise. */
int smc_simulate(smc_ctx *ctx, int precision, uint64_t seed, uint64_t traj_begin,
                 uint64_t n_traj, double confidence, const smc_sim_out *out, void *stream);

/* Diagnostic: replays given paths through the compiled monitor on the GPU
 * (single-network models, atoms as loaded) -- the same device code that the
 * SSA kernel steps after every event.  Host arrays: len[n_paths] states per
 * path (>= 1), x[sum len][S] counts, t[sum len] entry times (t[0] = 0,
 * non-decreasing), tmin[n_paths] lower bound of the next entry time after
 * the last state, closed[n_paths] = 1 when the path has no further state.
 * Outputs: verdict[n_paths] (0 undetermined, 1 false, 2 true) and
 * decided_at[n_paths]: 2k when fixed by state k, 2k+1 when fixed by the
 * entry time of state k+1 (or the end of the path), -1 if undetermined. */
int smc_monitor_replay(smc_ctx *ctx, int n_paths, const int32_t *len, const int32_t *x,
                       const double *t, const double *tmin, const uint8_t *closed,
                       int32_t *verdict, int64_t *decided_at);

/* Allocation-free variant of smc_simulate (the paper has no counterpart:
 * this serves callers that must not allocate device memory when they run,
 * for example code whose device memory is owned by another allocator, or a
 * loop that must not block in cudaMalloc / cudaFree).
 *
 * Same arguments and outputs as smc_simulate; the caller passes the outputs
 * in *out (device pointers, counts required).  Instead of the context's own
 * work-queue buffers, the SSA kernel uses a fixed device array of the
 * library (SMC_NOALLOC_MAX_INSTANCES 64-bit queue counters plus two 32-bit
 * words, about 32 KiB, held by every GPU that loads the library until the
 * process exits).  The call allocates nothing:
 *  - the context's model tables must already be on the device: call
 *    smc_simulate or smc_estimate once after loading the model and property
 *    (otherwise SMC_E_STATE);
 *  - more than SMC_NOALLOC_MAX_INSTANCES instances: SMC_E_INVALID_ARG;
 *  - the first call on a device looks up the array's device address
 *    (cudaGetSymbolAddress) and caches it; make that first call before any
 *    stream capture;
 *  - every call on a device shares the array; each call resets the counters
 *    it uses before its kernel runs, so consecutive calls are independent,
 *    but calls whose work overlaps on the GPU (other streams or host
 *    threads) race on the array and must be serialised by the caller. */
#define SMC_NOALLOC_MAX_INSTANCES 4096
int smc_simulate_noalloc(smc_ctx *ctx, int precision, uint64_t seed, uint64_t traj_begin,
                         uint64_t n_traj, double confidence, const smc_sim_out *out, void *stream);

/* ---- surrogate control variate ----------------------------------------------
 * Not in the paper: a learned predictor g(state at t_c) of P(phi | prefix),
 * used as a control variate.  The plain estimator of Sec. 3.3 stays the
 * reference: for any fixed g and beta the control-variate estimate is
 * unbiased. */

/* smc_simulate with a checkpoint snapshot: for each trajectory, snap = 0 and
 * x_snap = the state occupied at time t_snap, or snap = 1 when the verdict
 * was fixed before t_snap (verdict in out->verdict).  stop_at_snap != 0
 * stops every trajectory at its snapshot (prefix-only run; those are not
 * counted in out->counts and get status 2).  Device arrays: snap
 * [n_inst][n_traj] (uint8), x_snap [n_inst][n_traj][S_max] (int32), and
 * optionally e_snap [n_inst][n_traj] (uint32, may be null): the events up to
 * the snapshot, or up to the verdict when it was fixed before t_snap (what a
 * prefix-only run of that trajectory costs).  out->verdict must be given.
 * Does not synchronise. */
int smc_simulate_snapshot(smc_ctx *ctx, int precision, uint64_t seed, uint64_t traj_begin,
                          uint64_t n_traj, double t_snap, int stop_at_snap, const smc_sim_out *out,
                          uint8_t *snap, int32_t *x_snap, uint32_t *e_snap, void *stream);

/* Which quantities the snapshot features carry (single-network contexts;
 * not in the paper): the counts of n_species chosen species (species[i] in
 * [0, S), in that order; n_species = 0: every species, the default), the
 * time, then, if with_rates != 0, ln c_k - ref_k for every reaction k, with
 * ref = log_rate_ref (host [R], copied) or, when it is NULL, the mean of
 * ln c_k over the loaded instances (the default).  A context holding one
 * held-out instance of a family passes the family's reference, so that its
 * rate features match the ones the network was trained on.  At most 16
 * features in all.  Reset to the default by every model load.
 * Errors: STATE (no model), UNSUPPORTED (batched networks, more than 16
 * features), INVALID_ARG (index out of range, null list with n_species > 0,
 * a non-finite reference). */
int smc_set_features(smc_ctx *ctx, const int32_t *species, int n_species, int with_rates,
                     const double *log_rate_ref);

/* Features of snapshots (single-network contexts), as smc_set_features
 * chose them: row (m, k) of feat [n_inst * n_traj][F] (FP32, device), F =
 * Fs + 1 + (R or 0) = the chosen species' counts / x_scale (Fs values),
 * t_snap / t_scale, then the log-rate features of instance m.  x_scale: host
 * [Fs]. */
int smc_snapshot_features(smc_ctx *ctx, uint64_t n_traj, const int32_t *x_snap, double t_snap,
                          const float *x_scale, float t_scale, float *feat, void *stream);

/* The network: n_in (<= 16) -> 128 -> 128 -> 128 -> 1, ReLU, logistic
 * output; BF16 tensor-core (tcgen05) kernels with FP32 accumulation, FP32
 * master weights (SMC_MLP_NPARAM floats: W1[128][16], b1, W2[128][128], b2,
 * W3[128][128], b3, w4[128], b4), Adam.  Activations and deltas are rounded
 * to BF16 where they are stored (after the ReLU, after the mask); biases,
 * w4 and the logit stay FP32. */
#define SMC_MLP_NPARAM 35329
#define SMC_MLP_MAX_BATCH 4194304
typedef struct smc_mlp smc_mlp;
int smc_mlp_create(smc_mlp **out, int device, int n_in, uint64_t seed); /* He-uniform init */
void smc_mlp_destroy(smc_mlp *mlp);
const char *smc_mlp_last_error(const smc_mlp *mlp);
int smc_mlp_get_params(smc_mlp *mlp, float *host_params);       /* [SMC_MLP_NPARAM] */
int smc_mlp_set_params(smc_mlp *mlp, const float *host_params);
/* Gradient of the mean binary cross-entropy over n <= SMC_MLP_MAX_BATCH rows
 * (device x [n][n_in], y [n] in {0,1}); host outputs.  The same kernel as
 * a training step: one fused launch (forward, backward and weight
 * gradients of each 128-row tile in shared and tensor memory, one partial
 * gradient per CTA) and a launch summing the partials. */
int smc_mlp_gradient(smc_mlp *mlp, const float *x, const float *y, int n, float *grad_host,
                     float *loss_host);
/* Adam training: epochs (<= 4096) x ceil(n / batch) steps, batch <=
 * SMC_MLP_MAX_BATCH, minibatches drawn with replacement (step k of the
 * call takes row hash(seed, k, i) mod n as its row i; counter-based, so
 * the steps are replayed as captured CUDA graphs).  Asynchronous on
 * `stream` (NULL: the network's own stream) unless loss_host is given:
 * [epochs] mean loss per epoch, after a synchronisation.  A tensor-core
 * wait that gave up (bounded, about a second) makes this and every later
 * call on the network return SMC_E_CUDA. */
int smc_mlp_train(smc_mlp *mlp, const float *x, const float *y, uint64_t n, int epochs, int batch,
                  float lr, uint64_t seed, float *loss_host, void *stream);
/* g[i] = network output for row i of x (device [n][n_in] -> device [n]):
 * one persistent launch over 128-row tiles on the tcgen05 tensor cores
 * (one CTA per SM holding all of its tensor memory for the layers'
 * accumulators), features rounded to BF16 as in training.  Asynchronous on `stream`.  Should a
 * launch give up waiting for its tensor-core operations (a bounded wait,
 * about a second), it leaves NaN in the rows of the tile it was on and
 * every later predict call on this network returns SMC_E_CUDA. */
int smc_mlp_predict(smc_mlp *mlp, const float *x, uint64_t n, float *g, void *stream);
/* The same, computing only rows with skip[i] == 0 (device uint8 [n], may be
 * NULL): other entries of g are left as they were (tiles whose rows all
 * skip are not computed).  Used for trajectories decided before the
 * checkpoint, whose control variate is their verdict. */
int smc_mlp_predict_masked(smc_mlp *mlp, const float *x, uint64_t n, const uint8_t *skip, float *g,
                           void *stream);

/* Control-variate estimate for a single-instance context (two-phase
 * sampling; the network's inputs must be the snapshot features as
 * smc_set_features chose them, else INVALID_ARG): n_full trajectories run to their verdict Y, n_prefix further
 * trajectories only to t_snap; G = Y when the verdict was fixed before t_snap,
 * else G = g(snapshot features).  p_hat = mean_full(Y - beta G) +
 * beta mean_all(G), unbiased for any fixed beta.  Var is estimated from the
 * samples, n_eff = p_hat (1 - p_hat) / Var (n_eff = n_full while the full
 * runs hold only one verdict, as Fig. 2 treats p_hat = 0 or 1), and
 * [lo, hi] is Eq. 4 at n_eff.
 * The sample sizes grow (cost-optimal split between full and prefix runs,
 * with the events per full run and per prefix run measured on the full
 * runs) until n_eff >= Wilson_sample(p', half_width) with p' = p_hat +-
 * half_width as in Fig. 2; prefix runs are drawn only while they lower the
 * cost of the target variance (they do when the prefix's share of a run's
 * cost is below the share of Var(Y) that G explains).  Prefix runs use
 * trajectory indices from 2^31 up, full runs below 2^31.  x_scale [S]
 * (host), t_scale: feature scaling as in smc_snapshot_features; pilot: the
 * least first sample of full runs (>= 2; at least Fig. 2's first batch,
 * Wilson_sample(1, half_width)); later iterations go straight to the
 * cost-optimal sizes (at most 1024x growth).  Device buffers are kept in
 * the context for later calls. */
typedef struct {
    double p_hat, lo, hi;
    double n_eff;      /* p_hat (1 - p_hat) / var, or n_full (one verdict only) */
    double var;        /* estimated variance of p_hat */
    double beta;
    uint64_t n_full, n_prefix;
    uint64_t events_full, events_prefix; /* reactions fired by each sample */
    int32_t iterations, status;
} smc_cv_result;
int smc_estimate_cv(smc_ctx *ctx, smc_mlp *mlp, double confidence, double half_width, uint64_t seed,
                    int precision, double t_snap, const float *x_scale, float t_scale, double beta,
                    uint64_t pilot, smc_cv_result *out);

/* The natural logarithm used by the FP64 path for tau = -ln(u) / a_0
 * (Eq. 2a), evaluated on the integer pipes (GB300 runs FP64 arithmetic at
 * 1/64 of the FP32 rate): a table-driven method after Tang (ACM TOMS 16,
 * 1990) with an exact argument reduction and a 128-bit fixed-point sum,
 * within 0.502 ulp (correctly rounded but for values within ~2^-9 ulp of a
 * rounding midpoint); zero, negative, subnormal and non-finite arguments go
 * to the FP64 library logarithm.  Diagnostic entry point (tests).
 * u, out: device arrays of n doubles, caller-owned; out[i] = ln(u[i]),
 * enqueued on `stream` (0: the context's stream).  Errors: INVALID_ARG for
 * null pointers with n > 0, CUDA for a failed launch. */
int smc_log_fp64(smc_ctx *ctx, const double *u, uint64_t n, double *out, void *stream);

/* The division of the same step, tau = (-ln u) / a_0, on the integer pipes:
 * out[i] = num[i] / den[i] rounded to nearest-even, bit for bit the IEEE-754
 * binary64 quotient for every input (positive normal operands with a normal
 * quotient take the integer path, the rest the FP64 division).  Diagnostic
 * entry point (tests).  num, den, out: device arrays of n doubles, caller-
 * owned, enqueued on `stream` (0: the context's stream).  Errors:
 * INVALID_ARG for null pointers with n > 0, CUDA for a failed launch. */
int smc_div_fp64(smc_ctx *ctx, const double *num, const double *den, uint64_t n, double *out, void *stream);

/* Host utilities (no GPU needed). */
double smc_normal_quantile(double p);                           /* Phi^{-1}(p) */
int smc_wilson_interval(uint64_t yes, uint64_t n, double confidence, double *lo,
                        double *hi);                            /* Eq. 4 */
double smc_wilson_sample(double p, double half_width, double confidence); /* Eq. 5 */

/* One step of the iterative sample-size procedure of Fig. 2 (Sec. 3.3.2),
 * the decision smc_estimate takes between its batches, for callers that run
 * the batches themselves (e.g. several processes, each running a slice of
 * every batch and summing the counts).  Host only, no GPU needed.
 *
 *  sampling   SMC_ITERATIVE, SMC_CONSERVATIVE or SMC_FIXED_N;
 *  fixed_n    the batch of SMC_FIXED_N (1 .. 2^32-1), unused otherwise;
 *  confidence in (0, 1); half_width = epsilon of Eq. 5, in (0, 0.5) (unused
 *             for SMC_FIXED_N);
 *  yes, n     cumulative counts so far: verdicts true, verdicts decided
 *             (n <= n_tot; trajectories stopped by the event budget are in
 *             n_tot but not in n);
 *  n_tot      trajectories launched so far (0 before the first batch);
 *  *next      (out) trajectories to launch next, 0 = stop:
 *               n_tot = 0: fixed_n, ceil(Wilson_sample(0.5)) or
 *                          ceil(Wilson_sample(1)) (Eq. 5) by mode;
 *               else, SMC_ITERATIVE: p = yes / n (0 when n = 0),
 *                          p' = p + eps if p <= 1/2, else p - eps,
 *                          max(0, ceil(Wilson_sample(p')) - n_tot);
 *               else 0 (one batch).
 * Returns SMC_OK, or SMC_E_INVALID_ARG (bad mode or argument, yes > n,
 * n > n_tot, null next). */
int smc_fig2_next_batch(int sampling, uint64_t fixed_n, double confidence, double half_width,
                        uint64_t yes, uint64_t n, uint64_t n_tot, uint64_t *next);

#ifdef __cplusplus
}
#endif
#endif /* SMC_H */
