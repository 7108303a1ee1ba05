// smc_internal.h -- layouts shared by the host side of the library and its
// CUDA kernels: the compiled monitor program, the per-instance model table
// ("blob") staged into shared memory, and the kernel parameter block.
#pragma once
#include <stdint.h>

// Natural logarithm of the FP64 path (table-driven, Tang 1990): buckets
// around F_j = 0.75 + j / 256, j = 0..192; table = G_j [193] (9-bit
// approximations of 1/F_j) | ln(1/G_j) high [193] | ln(1/G_j) low [193] |
// ln 2 high | ln 2 low | pad.  The high parts are multiples of 2^-42, so
// k ln2_high + ln(1/G_j) high is exact for |k| <= 1075.
#include "smc_fp64i.h"
#define SMC_LOGTAB_BYTES FP64I_LOG_BYTES
// per-warp scratch of the specialized kernel's cooperative tail (the end of
// its warp slice)
#define SMC_JIT_COOP_BYTES 64  // the FP64 path's log table (a multiple of 16 bytes)
#define SMC_MAX_UNITS 4   // temporal operators (monitor units) per formula
#define SMC_MAX_ATOMS 6   // distinct atoms (truth tables are 64-bit)
#define SMC_MAX_SPECIES 255
#define SMC_MAX_REACTIONS 255

// ---------------------------------------------------------------------------
// Monitor program.
//
// A formula is compiled into at most SMC_MAX_UNITS "units", each of the form
//     L  U[a,b]  ( P  and  N )
// anchored at time 0, where L, P, Q are state formulas over the atoms (held
// as 64-entry truth tables indexed by the atom bit vector) and N is either
// tt (nest = 0), F[0,d] Q (nest = 1) or G[0,d] Q (nest = 2); nest = 3 is the
// unit X[a,b] P (the next state is entered within [a, b] and satisfies P).
// F[a,b] psi is
// tt U[a,b] psi; G[a,b] psi is compiled as the unit F[a,b] (not psi) whose
// value the top-level table negates.  A bare state formula at the top level
// is the unit ff U[0,0] P (decided at the initial state).
//
// The top-level boolean structure is a table over the units' Kleene values
// (0 = undetermined, 1 = false, 2 = true), indexed by sum_u value_u * 3^u,
// giving 0 (undetermined), 1 (false) or 2 (true).
struct MonUnit {
    uint64_t L, P, Q;  // truth tables over the atom bit vector
    double a, b;       // window of the unit (entry time of a witness)
    double d;          // window [0, d] of the nested operator
    int32_t nest;      // 0 none, 1 F-nested, 2 G-nested, 3 next
    int32_t pad;
};

struct MonProg {
    int32_t n_units, n_atoms;
    int32_t unbounded;  // some window end is +inf: pessimistic rule at t_max
    int32_t has_lower;  // some unit window starts after 0
    double t_max;
    MonUnit u[SMC_MAX_UNITS];
    uint8_t table[81];  // 3^SMC_MAX_UNITS
    uint8_t pad2[23];
};
static_assert(sizeof(MonUnit) == 56, "MonUnit layout");
static_assert(sizeof(MonProg) % 16 == 0, "MonProg is copied in 16-byte words");

// ---------------------------------------------------------------------------
// Per-instance table ("blob"), 32-bit words, every section 2-word aligned.
//   hdr[0..15]: S, R, n_atoms, total_words, then word offsets of the sections:
enum BlobHdr {
    BH_S = 0, BH_R, BH_NA, BH_WORDS,
    BH_RATE_D,    // double [R]      stochastic rate constants
    BH_RATE_F,    // float  [R]      the same, rounded to FP32
    BH_REAC,      // u32    [R]      propensity word of reaction k (below)
    BH_ST_PTR,    // u32    [R+1]    CSR row pointers of the stoichiometry
    BH_ST,        // u32    [nnz]    species | (delta << 8) (delta signed)
    BH_DEP_PTR,   // u32    [R+1]    CSR row pointers of dep(j)
    BH_DEP,       // u32    [ndep]   propensity words of the k in dep(j)
    BH_AMASK,     // u32    [R]      atoms whose linear form reaction j changes
    BH_ATERM_PTR, // u32    [NA+1]   CSR row pointers of the atoms' terms
    BH_ATERM,     // u32    [nterm]  species | (coef << 8) (coef signed)
    BH_X0,        // i32    [S]      initial counts
    BH_ATOM,      // u32    [NA][6]  atom record (below)
    BH_DENSE,     // u32    [R][2]   small networks only (else offset 0): the
                  //                 net changes of species 0..7 as int8 bytes
    BH_FACT_PTR,  // u32    [R+1]    CSR row pointers of the rate-law factors
    BH_FACT,      // u32    [nf]     species | (power << 8) of factor q
    BH_FACT_D,    // double [nf][4]  a0, a1, b0, b1 of factor q
    BH_FACT_F,    // float  [nf][4]  the same, rounded to FP32
    BH_EXPR,      // u32    [nt][4]  arithmetic atoms' tokens: kind | arg << 8, 0, value (double)
    BH_COUNT = 26
};
// The atom operators and arithmetic-atom tokens of include/smc.h, repeated
// (identical definitions) for the run-time compiled kernels, which cannot
// include that host header.
#define SMC_OP_LT 0
#define SMC_OP_LE 1
#define SMC_OP_GE 2
#define SMC_OP_GT 3
#define SMC_OP_EQ 4
#define SMC_OP_NE 5
#define SMC_TOK_SPECIES 0
#define SMC_TOK_CONST 1
#define SMC_TOK_ADD 2
#define SMC_TOK_SUB 3
#define SMC_TOK_MUL 4
#define SMC_TOK_DIV 5
#define SMC_TOK_SQRT 6
#define SMC_TOK_POWI 7
#define SMC_EXPR_MAX_DEPTH 8
// An arithmetic atom's record has word 0 = SMC_ATOM_EXPR, then op, the
// word offset of its tokens within BH_EXPR, the token counts of the left
// and right programs, 0.
#define SMC_ATOM_EXPR 0xFFFFFFFEu
// Rate-law factors: reaction k's propensity is c_k h_k(x) times, for each of
// its factors q in order, (a0 + a1 x^n) / (b0 + b1 x^n) with x the count of
// the factor's species; propensity words of reactions with factors carry
// bit 25 (SMC_PW_FACT).
#define SMC_PW_FACT (1u << 25)
#define SMC_MAX_FACTORS_PER_REACTION 2
#define SMC_MAX_FACTOR_POWER 4
// Small networks (S <= 8, R <= 8, |v_ji| <= 127) are stepped with warp-uniform
// loops: every propensity recomputed per event, selection on the prefix sums
// kept in registers, stoichiometry from the dense byte rows.
#define SMC_SMALL_MAX 8
// Atom record (6 words): [0] the single term species | coef << 8, or
// 0xFFFFFFFF when the atom has several terms (then the ATERM rows hold
// them); [1] neg (0/1); [2..3] lo and [4..5] hi (int64): the atom holds iff
// (lo <= L <= hi) xor neg, L = sum of coef * x over its terms.
// Propensity word: k | ra << 8 | rb << 16 | homo << 24.  Species index S is
// a constant-1 column of the lane state, so every mass-action propensity
// (Sec. 2.2) is a_k = c_k h with h = x_ra (x_rb - homo) >> homo:
// 1 (ra = rb = S), x_a (rb = S), x_a x_b, or x_a (x_a - 1) / 2 (homo = 1).

// ---------------------------------------------------------------------------
// Kernel parameters of the persistent SSA kernel.
struct SsaParams {
    const uint32_t *blobs;       // all instance tables, concatenated
    const uint64_t *blob_off;    // word offset of instance m's table
    const int32_t *inst_list;    // instances served by this launch
    int32_t n_list;
    int32_t n_inst;              // instances in the context
    const uint64_t *tbegin;      // [n_inst] first trajectory index
    const uint64_t *tend;        // [n_inst] one past the last index
    uint64_t u_begin, u_end;     // the range of every instance when uniform
    int32_t uniform;             // 1: ignore tbegin / tend
    unsigned long long *tnext;   // [n_inst] work queue (starts at tbegin)
    unsigned int *cursor;        // instance cursor (starts at 0)
    unsigned int *ticket;        // blocks finished (starts at 0)
    const MonProg *prog;
    const uint64_t *logtab;      // FP64 path: ln table (SMC_LOGTAB_BYTES, layout of smc_fp64i.h)
    int32_t logtab_bytes;        // its shared-memory footprint (0: mixed path)
    uint32_t rk0[10], rk1[10];   // Philox round keys
    uint64_t budget;             // max reactions per trajectory
    uint32_t renorm_mask;        // mixed path: renormalise when (e & mask) == 0
    int32_t refill;              // refill when >= refill lanes are idle
    int32_t s_max, r_max;        // per-lane state area
    int32_t tc_bytes;            // per-warp candidate clocks (0: no nested unit)
    int32_t warp_bytes;          // shared memory per warp
    // outputs
    unsigned long long *counts;  // [n_inst][4] yes, n, events, budget hits
    double *wilson;              // [n_inst][3] or null
    double z;                    // normal quantile for the Wilson epilogue
    uint8_t *o_verdict;          // per-trajectory outputs or null
    uint8_t *o_status;
    uint64_t *o_events;
    double *o_tfinal;
    int32_t *o_xfinal;
    uint64_t out_base;           // trajectory index of output column 0
    uint64_t out_stride;         // columns per instance row
    int32_t x_stride;            // species per x_final / x_snap row
    // checkpoint snapshot (surrogate control variate): the state occupied at
    // t_snap is written to o_xsnap and o_snap = 0; a trajectory decided
    // before t_snap gets o_snap = 1.  snap_mode 2 stops every trajectory at
    // its snapshot (prefix-only run; such trajectories are not counted).
    int32_t snap_mode;           // 0 none, 1 snapshot, 2 snapshot and stop
    double t_snap;
    uint8_t *o_snap;             // [n_inst][out_stride]
    int32_t *o_xsnap;            // [n_inst][out_stride][x_stride]
    uint32_t *o_esnap;           // [n_inst][out_stride] events up to the snapshot
                                 // (or to the verdict, if fixed before t_snap); may be null
    // generic kernel, networks of more than 16 reactions: 1 = selection by
    // the running sums at every 16th reaction (the warp slice then holds
    // SMC_SEL_BLOCKS(r_max) of them per lane after the propensities), 0 =
    // linear scan
    int32_t sel_block;
    // expected cost of a trajectory per instance (or null): warps that
    // have run out of fresh instances join the one with the most work left,
    // trajectories left x cost
    const float *inst_cost;
    // trace monitor (smc_nest.h; formulas nested beyond the units above):
    // when nest is set the units are unused, and each lane records its
    // trajectory's positions (at most tr_cap) in tr_t / tr_w, position m of
    // lane l = blockIdx.x * blockDim.x + threadIdx.x at l * tr_cap + m (a
    // lane's positions contiguous: its evaluation scans them in order):
    // entry times; atom bits | entering reaction << 24.  tr_m: the
    // evaluator's memo, slot k's cell for position m of lane l at
    // (l * n_slots + k) * tr_cap + m (nest->n_slots slots; null if none)
    const struct NestProg *nest;
    double *tr_t;
    uint32_t *tr_w;
    uint32_t *tr_m;
    uint32_t tr_cap;
};
#define SMC_SEL_BLOCK 16
#define SMC_SEL_BLOCKS(r) (((r) + SMC_SEL_BLOCK - 1) / SMC_SEL_BLOCK)

// Monitor replay (tests): runs the compiled monitor over given paths.
struct ReplayParams {
    const MonProg *prog;
    const int32_t *coef;     // [n_atoms][S] atom coefficients (compiled order)
    const int64_t *athr;     // [n_atoms][2]
    uint32_t aneg;
    int32_t S;
    int32_t n_paths;
    const int32_t *len;      // [n_paths] states per path
    const int64_t *off;      // [n_paths] first state of each path
    const int32_t *x;        // [total][S]
    const double *t;         // [total]
    const double *tmin;      // [n_paths] entry time bound after the last state
    const uint8_t *closed;   // [n_paths]
    int32_t *verdict;        // [n_paths] 0 undetermined, 1 false, 2 true
    int64_t *decided_at;     // [n_paths] 2k / 2k+1 decision point or -1
    const struct NestProg *nest;  // trace monitor instead of the units (or null)
    uint32_t *w;             // [total] scratch: atom bits per state (trace monitor)
};

#if defined(__cplusplus) && !defined(__CUDACC_RTC__)  // host code only (not in run-time compilation)
extern "C++" {
// host launch wrappers (smc_kernels.cu)
// ext: kernel variant, bit 0 the model uses rate-law factors or arithmetic
// atoms, bit 1 the trace monitor (SsaParams::nest)
int smc_launch_ssa(int plain, int ext, const SsaParams &p, int grid, int block, int smem_bytes,
                   void *stream);
const char *smc_kernel_error();  // text of the last failed launch wrapper's error
int smc_ssa_max_blocks_per_sm(int plain, int ext, int block, int smem_bytes, int *out);
int smc_ssa_set_smem_limit(int plain, int ext, int smem_bytes);
int smc_launch_queue_init(const SsaParams &p, void *stream);
int smc_launch_replay(const ReplayParams &p, void *stream);
int smc_launch_log_batch(const uint64_t *tab, const double *u, uint64_t n, double *out, void *stream);
int smc_launch_div_batch(const double *num, const double *den, uint64_t n, double *out, void *stream);
int smc_launch_snapshot_features(uint64_t n_rows, uint64_t n_traj, int Fs, const int32_t *sidx, int R,
                                 int x_stride, const int32_t *x_snap, const float *x_scale, float t_feat,
                                 const float *lograte, float *feat, void *stream);
int smc_launch_cv_sums(uint64_t n, const uint8_t *y, const uint8_t *snap, const float *g, const uint32_t *e_pre,
                       int prefix, double *sums, void *stream);
// model-specialized kernels (smc_jit.cpp): the same contract as the three
// above, for a kernel handle returned by smc::jit_compile
int smc_jit_set_smem_limit(void *kernel, int smem_bytes);
int smc_jit_max_blocks_per_sm(void *kernel, int block, int smem_bytes, int *out);
int smc_jit_launch(void *kernel, const SsaParams &p, int grid, int block, int smem_bytes, void *stream);
// fixed scratch of smc_simulate_noalloc (see smc_kernels.cu)
#define SMC_NOALLOC_MAX_DEVICES 64
int smc_noalloc_scratch(int device, unsigned long long **queue, unsigned int **sync);
}
#endif
