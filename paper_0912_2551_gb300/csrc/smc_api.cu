// smc_api.cu -- the C ABI (include/smc.h): context, model and property
// loading, the iterative Wilson procedure (Fig. 2) on the host, and the
// launches of the persistent SSA kernel.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "../../include/smc.h"
#include "smc_compile.h"
#include "smc_internal.h"
#include "smc_jit.h"
#include "smc_mlp.h"
#include "smc_cme.h"

namespace {

// Launch shape of one size class of instances.
struct Shape {
    int warps = 4;       // warps per block
    int blocks_sm = 0;   // blocks per SM (0 = as many as fit)
    int refill = 1;      // refill threshold
    bool tuned = false;
};

struct SizeClass {
    std::vector<int32_t> inst;  // instance ids
    int32_t *d_list = nullptr;
    int s_max = 0, r_max = 0, blob_words = 0;
    Shape shape[2];             // [plain]
};

}  // namespace

struct smc_ctx {
    int device = 0;
    int n_sm = 0;
    size_t smem_optin = 0;
    cudaStream_t stream = nullptr;
    std::string err;

    // model (host copies)
    bool have_model = false;
    bool batch = false;
    int n_inst = 0;
    std::vector<int> S, R;
    std::vector<size_t> reac_off, st_off, rate_off, x0_off;
    std::vector<int32_t> reactants, stoich, x0;
    std::vector<double> rates;
    int s_max = 0;
    // rate-law factors (smc_load_rate_factors), shared by all instances
    std::vector<int32_t> f_reac, f_spec, f_pow;
    std::vector<double> f_par;

    // property
    bool have_prop = false;
    MonProg prog;
    // trace monitor (formulas nested beyond the monitor's units, smc_nest.h)
    bool nest_mode = false;
    NestProg nest{};
    NestProg *d_nest = nullptr;
    uint32_t trace_cap = 4096;          // positions recorded per lane
    double *d_tr_t = nullptr;           // [lanes][trace_cap] entry times
    uint32_t *d_tr_w = nullptr;         // [lanes][trace_cap] atom bits | reaction << 24
    uint32_t *d_tr_m = nullptr;         // [lanes][slots][trace_cap] evaluator memo
    size_t tr_lanes = 0;                // lanes the buffers hold
    int tr_slots = 0;                   // memo slots they hold
    std::vector<int> used_atoms;
    int n_atoms = 0;
    bool per_instance_bound = false;
    std::vector<int32_t> atom_op;
    std::vector<double> atom_bound;   // [n_atoms] or [n_inst][n_atoms]
    std::vector<int32_t> atom_coef;   // concatenated per instance [n_atoms][S_m]
    // arithmetic atoms (smc_set_atom_expression), [n_atoms]; op < 0: linear
    struct AtomExpr {
        int op = -1;
        std::vector<smc_token> lhs, rhs;
    };
    std::vector<AtomExpr> atom_expr;
    std::vector<size_t> coef_off;

    // device state
    bool dirty = true;
    uint32_t *d_blobs = nullptr;
    uint64_t *d_blob_off = nullptr;
    MonProg *d_prog = nullptr;
    std::vector<SizeClass> classes;  // instances grouped by reaction count
    SizeClass single;                // every instance in one launch
    bool use_single[2] = {false, false};
    bool tuned[2] = {false, false};
    // autotuner results of the last tuned model structure, per precision:
    // reused when a model of the same structure is loaded again
    struct TuneMemo {
        bool valid = false;
        std::vector<int64_t> sig;
        std::vector<Shape> cls;
        Shape single;
        bool use_single = false;
    } memo[2];
    unsigned long long *d_trial = nullptr;  // autotuner counts
    float *d_cost = nullptr;                // expected events per trajectory, per instance (from the trials)
    bool have_cost = false;
    uint64_t *d_tbegin = nullptr, *d_tend = nullptr;
    unsigned long long *d_tnext = nullptr;
    unsigned int *d_sync = nullptr;  // cursor, ticket
    unsigned long long *d_counts = nullptr;
    double *d_wilson = nullptr;
    uint64_t *h_range = nullptr;     // pinned [2][n_inst]
    unsigned long long *h_counts = nullptr;
    double *h_wilson = nullptr;
    uint8_t *d_record = nullptr;
    uint64_t record_n = 0, record_valid = 0;
    float *d_feat_aux = nullptr;  // feature scales, species indices and log-rate features
    size_t feat_aux_n = 0;
    // the snapshot features (smc_set_features): species (empty: all), rate
    // features on or off, their reference (empty: the mean over the instances)
    std::vector<int32_t> feat_species;
    int feat_rates = 1;
    std::vector<double> feat_ref;
    uint64_t *d_logtab = nullptr;  // table of the FP64 path's logarithm (lives with the context)
    // control-variate estimator's buffers, grown on demand and kept (a
    // cudaFree per call would synchronise the device)
    struct CvBuf {
        uint8_t *y = nullptr, *snap = nullptr;
        int32_t *x = nullptr;
        uint32_t *e = nullptr;
        float *feat = nullptr, *g = nullptr;
        uint64_t *counts = nullptr;
        double *sums = nullptr;
        uint64_t cap = 0;
        int s_cap = 0, f_cap = 0;
        void release()
        {
            cudaFree(y); cudaFree(snap); cudaFree(x); cudaFree(e); cudaFree(feat); cudaFree(g);
            cudaFree(counts); cudaFree(sums);
            *this = CvBuf();
        }
    } cv;

    // options
    uint64_t budget = 1ull << 24;
    int renorm_log2 = 8;
    int autotune = 1;
    bool explicit_shape = false;  // a shape option was set: do not tune
    int warps = 4;
    int blocks_sm = 0;
    int refill = 1;
    int record = 0;
    int jit = 1;                  // model-specialized kernels when eligible
    int selection = 0;            // SMC_OPT_SELECTION
    // specialized kernels of the loaded structure (null: the generic ones run)
    smc::JitKernels jit_k;
    bool jit_ready = false;
    bool ext = false;             // rate-law factors or arithmetic atoms in use (generic kernel variant)
    std::string jit_why;          // why they are not in use
};

namespace {

int fail(smc_ctx *c, int code, const std::string &msg)
{
    if (c) c->err = msg;
    return code;
}

#define CK(call)                                                                          \
    do {                                                                                  \
        cudaError_t e_ = (call);                                                          \
        if (e_ != cudaSuccess)                                                            \
            return fail(ctx, e_ == cudaErrorMemoryAllocation ? SMC_E_OOM : SMC_E_CUDA,    \
                        std::string(#call) + ": " + cudaGetErrorString(e_));              \
    } while (0)

template <class T>
void dfree(T *&p)
{
    if (p) cudaFree((void *)p);
    p = nullptr;
}

void free_device(smc_ctx *ctx)
{
    dfree(ctx->d_blobs);
    dfree(ctx->d_blob_off);
    dfree(ctx->d_prog);
    dfree(ctx->d_nest);
    dfree(ctx->d_tr_t);
    dfree(ctx->d_tr_w);
    dfree(ctx->d_tr_m);
    ctx->tr_lanes = 0;
    ctx->tr_slots = 0;
    for (auto &c : ctx->classes) dfree(c.d_list);
    ctx->classes.clear();
    dfree(ctx->single.d_list);
    ctx->single = SizeClass();
    dfree(ctx->d_trial);
    dfree(ctx->d_cost);
    ctx->have_cost = false;
    ctx->use_single[0] = ctx->use_single[1] = false;
    ctx->tuned[0] = ctx->tuned[1] = false;
    dfree(ctx->d_tbegin);
    dfree(ctx->d_tend);
    dfree(ctx->d_tnext);
    dfree(ctx->d_sync);
    dfree(ctx->d_counts);
    dfree(ctx->d_wilson);
    dfree(ctx->d_record);
    dfree(ctx->d_feat_aux);
    ctx->feat_aux_n = 0;
    if (ctx->h_range) cudaFreeHost(ctx->h_range);
    if (ctx->h_counts) cudaFreeHost(ctx->h_counts);
    if (ctx->h_wilson) cudaFreeHost(ctx->h_wilson);
    ctx->h_range = nullptr;
    ctx->h_counts = nullptr;
    ctx->h_wilson = nullptr;
    ctx->record_n = ctx->record_valid = 0;
}

// AS241 (Wichura 1988, PPND16): the standard normal quantile to about 1e-16,
// three rational approximations (central, intermediate and far tail).
double as241(double p)
{
    if (!(p > 0.0 && p < 1.0)) return std::nan("");
    const double q = p - 0.5;
    if (std::fabs(q) <= 0.425) {
        const double r = 0.180625 - q * q;
        const double num = (((((((2.5090809287301226727e+3 * r + 3.3430575583588128105e+4) * r +
                                 6.7265770927008700853e+4) * r + 4.5921953931549871457e+4) * r +
                               1.3731693765509461125e+4) * r + 1.9715909503065514427e+3) * r +
                             1.3314166789178437745e+2) * r + 3.3871328727963666080e0);
        const double den = (((((((5.2264952788528545610e+3 * r + 2.8729085735721942674e+4) * r +
                                 3.9307895800092710610e+4) * r + 2.1213794301586595867e+4) * r +
                               5.3941960214247511077e+3) * r + 6.8718700749205790830e+2) * r +
                             4.2313330701600911252e+1) * r + 1.0);
        return q * num / den;
    }
    double r = q < 0.0 ? p : 1.0 - p;
    r = std::sqrt(-std::log(r));
    double z;
    if (r <= 5.0) {
        r -= 1.6;
        const double num = (((((((7.74545014278341407640e-4 * r + 2.27238449892691845833e-2) * r +
                                 2.41780725177450611770e-1) * r + 1.27045825245236838258e0) * r +
                               3.64784832476320460504e0) * r + 5.76949722146069140550e0) * r +
                             4.63033784615654529590e0) * r + 1.42343711074968357734e0);
        const double den = (((((((1.05075007164441684324e-9 * r + 5.47593808499534494600e-4) * r +
                                 1.51986665636164571966e-2) * r + 1.48103976427480074590e-1) * r +
                               6.89767334985100004550e-1) * r + 1.67638483018380384940e0) * r +
                             2.05319162663775882187e0) * r + 1.0);
        z = num / den;
    } else {
        r -= 5.0;
        const double num = (((((((2.01033439929228813265e-7 * r + 2.71155556874348757815e-5) * r +
                                 1.24266094738807843860e-3) * r + 2.65321895265761230930e-2) * r +
                               2.96560571828504891230e-1) * r + 1.78482653991729133580e0) * r +
                             5.46378491116411436990e0) * r + 6.65790464350110377720e0);
        const double den = (((((((2.04426310338993978564e-15 * r + 1.42151175831644588870e-7) * r +
                                 1.84631831751005468180e-5) * r + 7.86869131145613259100e-4) * r +
                               1.48753612908506148525e-2) * r + 1.36929880922735805310e-1) * r +
                             5.99832206555887937690e-1) * r + 1.0);
        z = num / den;
    }
    return q < 0.0 ? -z : z;
}

double z_of(double confidence) { return as241(1.0 - (1.0 - confidence) / 2.0); }

// Eq. 5
double wilson_sample_real(double p, double eps, double z)
{
    const double e2 = eps * eps, v = p * (1.0 - p);
    return z * z * (v - 2.0 * e2 + std::sqrt(v * v + 4.0 * e2 * (p - 0.5) * (p - 0.5))) / (2.0 * e2);
}

uint64_t wilson_sample_n(double p, double eps, double z)
{
    const double n = std::ceil(wilson_sample_real(p, eps, z));
    return n < 1.0 ? 1 : (uint64_t)n;
}

// Fig. 2: the batch after n_tot launched trajectories with cumulative counts
// (yes, dec); 0 = stop.  The first batch is Eq. 5 at the mode's starting p.
uint64_t fig2_next(int sampling, uint64_t fixed_n, double eps, double z, uint64_t yes, uint64_t dec, uint64_t n_tot)
{
    if (n_tot == 0) {
        if (sampling == SMC_FIXED_N) return fixed_n;
        return wilson_sample_n(sampling == SMC_CONSERVATIVE ? 0.5 : 1.0, eps, z);
    }
    if (sampling != SMC_ITERATIVE) return 0;
    const double p_est = dec ? (double)yes / (double)dec : 0.0;
    const double p_prime = p_est <= 0.5 ? p_est + eps : p_est - eps;
    const uint64_t n_prime = wilson_sample_n(p_prime, eps, z);
    return n_prime > n_tot ? n_prime - n_tot : 0;
}

// Eq. 4 on the host (same operation order as the device epilogue).
void wilson_host(uint64_t yes, uint64_t n, double z, double *p_out, double *lo_out, double *hi_out)
{
    if (n == 0) { *p_out = std::nan(""); *lo_out = 0.0; *hi_out = 1.0; return; }
    const double dn = (double)n, p = (double)yes / dn, z2 = z * z;
    const double centre = p + z2 / (2.0 * dn);
    const double half = z * std::sqrt(p * (1.0 - p) / dn + z2 / (4.0 * dn * dn));
    const double den = 1.0 + z2 / dn;
    double lo = (centre - half) / den, hi = (centre + half) / den;
    if (yes == 0) lo = 0.0;
    if (yes == n) hi = 1.0;
    *p_out = p;
    *lo_out = std::max(0.0, lo);
    *hi_out = std::min(1.0, hi);
}

void round_keys(uint64_t seed, uint32_t rk0[10], uint32_t rk1[10])
{
    uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
    for (int r = 0; r < 10; ++r) {
        rk0[r] = k0;
        rk1[r] = k1;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
}

int validate_network(smc_ctx *ctx, int S, int R, const int32_t *reac, const int32_t *st)
{
    if (S < 1 || S > SMC_MAX_SPECIES || R < 1 || R > SMC_MAX_REACTIONS)
        return fail(ctx, SMC_E_INVALID_ARG, "species and reactions per network must be 1..255");
    for (int j = 0; j < R; ++j) {
        for (int s = 0; s < 2; ++s) {
            const int v = reac[2 * j + s];
            if (v < -1 || v >= S) return fail(ctx, SMC_E_INVALID_ARG, "reactant index out of range");
        }
        for (int i = 0; i < S; ++i) {
            const int d = st[(size_t)j * S + i];
            if (d > (1 << 22) || d < -(1 << 22))
                return fail(ctx, SMC_E_INVALID_ARG, "stoichiometric change out of range");
        }
    }
    return SMC_OK;
}

int validate_params(smc_ctx *ctx, int S, int R, const double *rates, const int32_t *x0)
{
    for (int j = 0; j < R; ++j)
        if (!(rates[j] >= 0.0) || !std::isfinite(rates[j]))
            return fail(ctx, SMC_E_INVALID_ARG, "rate constants must be finite and >= 0");
    for (int i = 0; i < S; ++i)
        if (x0[i] < 0) return fail(ctx, SMC_E_INVALID_ARG, "initial counts must be >= 0");
    return SMC_OK;
}

// The arithmetic atoms among the used atoms (views in used-atom order), and
// whether there is any.
std::vector<smc::AtomExprView> used_expr(const smc_ctx *ctx, bool &any)
{
    std::vector<smc::AtomExprView> v(ctx->used_atoms.size());
    any = false;
    for (size_t b = 0; b < v.size(); ++b) {
        const int a = ctx->used_atoms[b];
        if (a >= (int)ctx->atom_expr.size() || ctx->atom_expr[a].op < 0) continue;
        const auto &e = ctx->atom_expr[a];
        v[b].op = e.op;
        v[b].lhs = e.lhs.data();
        v[b].n_lhs = (int)e.lhs.size();
        v[b].rhs = e.rhs.data();
        v[b].n_rhs = (int)e.rhs.size();
        any = true;
    }
    return v;
}

// Model-specialized kernels: when every instance shares one structure
// (species, reactions, reactants, stoichiometry, monitored atoms and their
// thresholds), the structure is compiled into the kernel; rates and x0 stay
// data.  Otherwise (or without NVRTC) the generic kernels run.
void try_specialize(smc_ctx *ctx)
{
    ctx->jit_ready = false;
    ctx->jit_why.clear();
    if (!ctx->jit) { ctx->jit_why = "disabled by option"; return; }
    if (ctx->nest_mode) { ctx->jit_why = "the formula needs the trace monitor"; return; }
    const int n = ctx->n_inst, S = ctx->S[0], R = ctx->R[0], nu = (int)ctx->used_atoms.size();
    std::vector<int32_t> coef0((size_t)nu * S);
    std::vector<int64_t> lo0(nu), hi0(nu);
    std::vector<uint8_t> neg0(nu);
    for (int m = 0; m < n; ++m) {
        if (ctx->S[m] != S || ctx->R[m] != R) { ctx->jit_why = "instances differ in structure"; return; }
        if (m > 0 && (std::memcmp(ctx->reactants.data() + ctx->reac_off[m], ctx->reactants.data() + ctx->reac_off[0],
                                  sizeof(int32_t) * 2 * R) ||
                      std::memcmp(ctx->stoich.data() + ctx->st_off[m], ctx->stoich.data() + ctx->st_off[0],
                                  sizeof(int32_t) * (size_t)R * S))) {
            ctx->jit_why = "instances differ in structure";
            return;
        }
        for (int b = 0; b < nu; ++b) {
            const int a = ctx->used_atoms[b];
            if (a < (int)ctx->atom_expr.size() && ctx->atom_expr[a].op >= 0) continue;  // same for all
            const int32_t *c = ctx->atom_coef.data() + ctx->coef_off[m] + (size_t)a * S;
            const double bnd = ctx->per_instance_bound ? ctx->atom_bound[(size_t)m * ctx->n_atoms + a] : ctx->atom_bound[a];
            int64_t lo, hi;
            bool neg;
            smc::atom_threshold(ctx->atom_op[a], bnd, lo, hi, neg);
            if (m == 0) {
                std::memcpy(&coef0[(size_t)b * S], c, sizeof(int32_t) * S);
                lo0[b] = lo;
                hi0[b] = hi;
                neg0[b] = neg;
            } else if (std::memcmp(&coef0[(size_t)b * S], c, sizeof(int32_t) * S) || lo != lo0[b] || hi != hi0[b] ||
                       (uint8_t)neg != neg0[b]) {
                ctx->jit_why = "instances differ in their atoms";
                return;
            }
        }
    }
    smc::JitModel M;
    M.S = S;
    M.R = R;
    M.reactants = ctx->reactants.data() + ctx->reac_off[0];
    M.stoich = ctx->stoich.data() + ctx->st_off[0];
    M.n_atoms = nu;
    M.coef = coef0.data();
    M.lo = lo0.data();
    M.hi = hi0.data();
    M.neg = neg0.data();
    M.n_fact = (int)ctx->f_reac.size();
    M.f_reac = ctx->f_reac.data();
    M.f_spec = ctx->f_spec.data();
    M.f_pow = ctx->f_pow.data();
    M.f_par = ctx->f_par.data();
    bool any_expr = false;
    const std::vector<smc::AtomExprView> ev = used_expr(ctx, any_expr);
    M.expr = any_expr ? ev.data() : nullptr;
    const std::string header = smc::jit_model_header(M, ctx->jit_why);
    if (header.empty()) return;
    std::string err;
    if (smc::jit_compile(header, ctx->jit_k, err)) { ctx->jit_why = err; return; }
    smc::jit_layout(M, ctx->jit_k.delta_bytes, ctx->jit_k.rate_count);
    ctx->jit_ready = true;
}

// Builds the instance tables, size classes and work buffers on the device.
int prepare(smc_ctx *ctx)
{
    if (!ctx->have_model || !ctx->have_prop) return fail(ctx, SMC_E_STATE, "load a model and a property first");
    if (!ctx->dirty) return SMC_OK;
    CK(cudaSetDevice(ctx->device));
    free_device(ctx);
    const int n = ctx->n_inst, nu = (int)ctx->used_atoms.size();
    std::vector<uint32_t> all;
    std::vector<uint64_t> off(n);
    std::vector<int> words(n);
    std::vector<uint32_t> blob;
    for (int m = 0; m < n; ++m) {
        smc::InstanceModel M;
        M.S = ctx->S[m];
        M.R = ctx->R[m];
        M.reactants = ctx->reactants.data() + ctx->reac_off[m];
        M.stoich = ctx->stoich.data() + ctx->st_off[m];
        M.rates = ctx->rates.data() + ctx->rate_off[m];
        M.x0 = ctx->x0.data() + ctx->x0_off[m];
        M.n_fact = (int)ctx->f_reac.size();
        M.f_reac = ctx->f_reac.data();
        M.f_spec = ctx->f_spec.data();
        M.f_pow = ctx->f_pow.data();
        M.f_par = ctx->f_par.data();
        std::vector<int32_t> coef((size_t)nu * M.S), op(nu);
        std::vector<double> bnd(nu);
        for (int b = 0; b < nu; ++b) {
            const int a = ctx->used_atoms[b];
            std::memcpy(&coef[(size_t)b * M.S], ctx->atom_coef.data() + ctx->coef_off[m] + (size_t)a * M.S,
                        sizeof(int32_t) * M.S);
            op[b] = ctx->atom_op[a];
            bnd[b] = ctx->per_instance_bound ? ctx->atom_bound[(size_t)m * ctx->n_atoms + a]
                                             : ctx->atom_bound[a];
        }
        bool any_expr = false;
        const std::vector<smc::AtomExprView> ev = used_expr(ctx, any_expr);
        int rc = smc::build_blob(M, nu, coef.data(), op.data(), bnd.data(), any_expr ? ev.data() : nullptr, blob,
                                 ctx->err);
        if (rc) return rc;
        off[m] = all.size();
        words[m] = (int)blob.size();
        all.insert(all.end(), blob.begin(), blob.end());
    }
    // size classes by reaction count (each class gets its own launch shape)
    const int bounds[] = {8, 16, 32, 64, 128, 256};
    for (int bnd : bounds) {
        SizeClass c;
        for (int m = 0; m < n; ++m) {
            const int lo = (bnd == 8) ? 0 : bnd / 2;
            if (ctx->R[m] > lo && ctx->R[m] <= bnd) {
                c.inst.push_back(m);
                c.s_max = std::max(c.s_max, ctx->S[m]);
                c.r_max = std::max(c.r_max, ctx->R[m]);
                c.blob_words = std::max(c.blob_words, words[m]);
            }
        }
        if (!c.inst.empty()) ctx->classes.push_back(c);
    }
    for (int m = 0; m < n; ++m) {
        ctx->single.inst.push_back(m);
        ctx->single.s_max = std::max(ctx->single.s_max, ctx->S[m]);
        ctx->single.r_max = std::max(ctx->single.r_max, ctx->R[m]);
        ctx->single.blob_words = std::max(ctx->single.blob_words, words[m]);
    }
    CK(cudaMalloc(&ctx->d_blobs, all.size() * 4));
    CK(cudaMemcpy(ctx->d_blobs, all.data(), all.size() * 4, cudaMemcpyHostToDevice));
    CK(cudaMalloc(&ctx->d_blob_off, n * 8));
    CK(cudaMemcpy(ctx->d_blob_off, off.data(), n * 8, cudaMemcpyHostToDevice));
    CK(cudaMalloc(&ctx->d_prog, sizeof(MonProg)));
    CK(cudaMemcpy(ctx->d_prog, &ctx->prog, sizeof(MonProg), cudaMemcpyHostToDevice));
    if (ctx->nest_mode) {
        CK(cudaMalloc(&ctx->d_nest, sizeof(NestProg)));
        CK(cudaMemcpy(ctx->d_nest, &ctx->nest, sizeof(NestProg), cudaMemcpyHostToDevice));
    }
    std::vector<SizeClass *> all_classes;
    for (auto &c : ctx->classes) all_classes.push_back(&c);
    all_classes.push_back(&ctx->single);
    for (SizeClass *c : all_classes) {
        CK(cudaMalloc(&c->d_list, c->inst.size() * 4));
        CK(cudaMemcpy(c->d_list, c->inst.data(), c->inst.size() * 4, cudaMemcpyHostToDevice));
        for (int pl = 0; pl < 2; ++pl) {
            c->shape[pl].warps = ctx->warps;
            c->shape[pl].blocks_sm = ctx->blocks_sm;
            c->shape[pl].refill = ctx->refill;
        }
    }
    CK(cudaMalloc(&ctx->d_trial, (size_t)n * 4 * 8));
    CK(cudaMalloc(&ctx->d_cost, (size_t)n * 4));
    CK(cudaMalloc(&ctx->d_tbegin, n * 8));
    CK(cudaMalloc(&ctx->d_tend, n * 8));
    CK(cudaMalloc(&ctx->d_tnext, n * 8));
    CK(cudaMalloc(&ctx->d_sync, 16));
    CK(cudaMalloc(&ctx->d_counts, (size_t)n * 4 * 8));
    CK(cudaMalloc(&ctx->d_wilson, (size_t)n * 3 * 8));
    CK(cudaMallocHost(&ctx->h_range, (size_t)n * 2 * 8));
    CK(cudaMallocHost(&ctx->h_counts, (size_t)n * 4 * 8));
    CK(cudaMallocHost(&ctx->h_wilson, (size_t)n * 3 * 8));
    {
        bool any_expr = false;
        used_expr(ctx, any_expr);
        ctx->ext = any_expr || !ctx->f_reac.empty();
    }
    try_specialize(ctx);
    ctx->dirty = false;
    return SMC_OK;
}

// generic kernel variant: bit 0 rate-law factors / arithmetic atoms, bit 1
// the trace monitor
int kvar(const smc_ctx *ctx) { return (ctx->ext ? 1 : 0) | (ctx->nest_mode ? 2 : 0); }

// Trace monitor: recording buffers for `lanes` lanes of trace_cap positions
// and the evaluator's memo, 4 bytes per position and slot (grown, never
// shrunk, while the context's device state lives).  Called when a launch is
// planned, before any stream capture.
int ensure_trace(smc_ctx *ctx, size_t lanes)
{
    const int slots = ctx->nest.n_slots;
    if (ctx->tr_lanes >= lanes && ctx->d_tr_t && ctx->tr_slots >= slots) return SMC_OK;
    dfree(ctx->d_tr_t);
    dfree(ctx->d_tr_w);
    dfree(ctx->d_tr_m);
    ctx->tr_lanes = 0;
    ctx->tr_slots = 0;
    const size_t n = lanes * ctx->trace_cap;
    if (cudaMalloc(&ctx->d_tr_t, n * sizeof(double)) != cudaSuccess ||
        cudaMalloc(&ctx->d_tr_w, n * sizeof(uint32_t)) != cudaSuccess ||
        (slots > 0 && cudaMalloc(&ctx->d_tr_m, n * slots * sizeof(uint32_t)) != cudaSuccess)) {
        cudaGetLastError();
        dfree(ctx->d_tr_t);
        dfree(ctx->d_tr_w);
        dfree(ctx->d_tr_m);
        return fail(ctx, SMC_E_OOM, "trace monitor buffers (" + std::to_string(n * (12 + 4 * slots) >> 20) +
                                    " MiB): lower SMC_OPT_TRACE_CAP or the launch shape");
    }
    ctx->tr_lanes = lanes;
    ctx->tr_slots = slots;
    return SMC_OK;
}

// candidate clocks per warp: only formulas with a nested F / G keep them
int tc_bytes_of(const MonProg &prog)
{
    for (int u = 0; u < prog.n_units; ++u)
        if (prog.u[u].nest) return SMC_MAX_UNITS * 32 * 8;
    return 0;
}

// Whether the generic kernel selects by checkpointed running sums for class c
// (SMC_OPT_SELECTION).
bool blocked_selection(const smc_ctx *ctx, const SizeClass &c)
{
    return ctx->selection == 2 ? c.r_max > SMC_SEL_BLOCK : ctx->selection == 0 && c.r_max > 64;
}

// warp slice: x[(s_max + 1)][32] | tc | a[r_max][32] | (blocked selection)
// running sums at every 16th reaction [SMC_SEL_BLOCKS(r_max)][32]; the
// tables stay in global memory
int warp_bytes_of(const SizeClass &c, int plain, int tc_bytes, bool blocked)
{
    const int b = (c.s_max + 1) * 128 + tc_bytes +
                  (c.r_max + (blocked ? SMC_SEL_BLOCKS(c.r_max) : 0)) * 32 * (plain ? 8 : 4);
    return (b + 15) & ~15;
}

// One planned launch of the SSA kernel for a set of instances.
struct Launch {
    const SizeClass *c = nullptr;
    void *kernel = nullptr;  // model-specialized kernel, or null for the generic one
    int grid = 0, block = 0, smem = 0, warp_bytes = 0, tc_bytes = 0, refill = 1;
    bool blocked = false;    // generic kernel: checkpointed selection
};

// The instance partition in use for a precision: the size classes, or one
// launch over every instance (chosen by the autotuner).
std::vector<const SizeClass *> active_classes(const smc_ctx *ctx, int plain)
{
    std::vector<const SizeClass *> v;
    if (ctx->use_single[plain] && ctx->classes.size() > 1) v.push_back(&ctx->single);
    else
        for (const auto &c : ctx->classes) v.push_back(&c);
    return v;
}

// Launch geometry of class c with shape sh (sets the kernel's shared-memory
// limit; call outside stream capture).  Returns SMC_E_UNSUPPORTED if it does
// not fit.
int plan_class(smc_ctx *ctx, int plain, const SizeClass &c, const Shape &sh, Launch &L)
{
    L.c = &c;
    L.tc_bytes = tc_bytes_of(ctx->prog);
    // the specialized kernel keeps counts and propensities in registers: its
    // warp slice holds only the nested operators' candidate clocks
    L.kernel = ctx->jit_ready ? (plain ? ctx->jit_k.plain : ctx->jit_k.mixed) : nullptr;
    const int rate_bytes = (ctx->jit_k.rate_count * (plain ? 8 : 4) + 15) / 16 * 16;
    L.blocked = !L.kernel && blocked_selection(ctx, c);
    L.warp_bytes = L.kernel ? L.tc_bytes + rate_bytes + SMC_JIT_COOP_BYTES
                            : warp_bytes_of(c, plain, L.tc_bytes, L.blocked);
    L.block = 32 * sh.warps;
    L.smem = (int)sizeof(MonProg) + (plain ? SMC_LOGTAB_BYTES : 0) + (L.kernel ? ctx->jit_k.delta_bytes : 0) +
             sh.warps * L.warp_bytes;
    L.refill = sh.refill;
    if ((size_t)L.smem > ctx->smem_optin)
        return fail(ctx, SMC_E_UNSUPPORTED, "model tables do not fit in shared memory");
    const int set_rc =
        L.kernel ? smc_jit_set_smem_limit(L.kernel, L.smem) : smc_ssa_set_smem_limit(plain, kvar(ctx), L.smem);
    if (set_rc) return fail(ctx, SMC_E_CUDA, "cudaFuncSetAttribute failed");
    int per_sm = 0;
    const int occ_rc = L.kernel ? smc_jit_max_blocks_per_sm(L.kernel, L.block, L.smem, &per_sm)
                                : smc_ssa_max_blocks_per_sm(plain, kvar(ctx), L.block, L.smem, &per_sm);
    if (occ_rc || per_sm < 1) return fail(ctx, SMC_E_UNSUPPORTED, "no block of this shape fits on an SM");
    if (sh.blocks_sm > 0) per_sm = std::min(per_sm, sh.blocks_sm);
    L.grid = ctx->n_sm * per_sm;
    if (ctx->nest_mode) return ensure_trace(ctx, (size_t)L.grid * L.block);
    return SMC_OK;
}

// Queue reset + SSA kernel for one planned launch (stream operations only,
// so it may be captured in a CUDA graph).
int issue_class(smc_ctx *ctx, int plain, const SsaParams &common, const Launch &L, cudaStream_t s)
{
    SsaParams p = common;
    p.inst_list = L.c->d_list;
    p.n_list = (int)L.c->inst.size();
    p.refill = L.refill;
    p.s_max = L.c->s_max;
    p.r_max = L.c->r_max;
    p.tc_bytes = L.tc_bytes;
    p.warp_bytes = L.warp_bytes;
    p.sel_block = L.blocked ? 1 : 0;
    p.logtab = ctx->d_logtab;
    p.logtab_bytes = plain ? SMC_LOGTAB_BYTES : 0;
    if (ctx->nest_mode) {  // buffers as planned (launches on one stream, one after another)
        p.nest = ctx->d_nest;
        p.tr_t = ctx->d_tr_t;
        p.tr_w = ctx->d_tr_w;
        p.tr_m = ctx->nest.n_slots > 0 ? ctx->d_tr_m : nullptr;
        p.tr_cap = ctx->trace_cap;
    }
    if (smc_launch_queue_init(p, s))
        return fail(ctx, SMC_E_CUDA, std::string("queue init: ") + cudaGetErrorString(cudaGetLastError()));
    const int lrc = L.kernel ? smc_jit_launch(L.kernel, p, L.grid, L.block, L.smem, s)
                             : smc_launch_ssa(plain, kvar(ctx), p, L.grid, L.block, L.smem, s);
    if (lrc)
        return fail(ctx, SMC_E_CUDA,
                    std::string("ssa launch: ") + (L.kernel ? cudaGetErrorString(cudaGetLastError()) : smc_kernel_error()));
    return SMC_OK;
}

void fill_common(smc_ctx *ctx, SsaParams &p, uint64_t seed, double z, const smc_sim_out &out,
                 uint64_t out_base, uint64_t out_stride, bool uniform)
{
    std::memset(&p, 0, sizeof(p));
    p.blobs = ctx->d_blobs;
    p.blob_off = ctx->d_blob_off;
    p.n_inst = ctx->n_inst;
    p.tbegin = ctx->d_tbegin;
    p.tend = ctx->d_tend;
    p.uniform = uniform;
    p.u_begin = out_base;
    p.u_end = out_base + out_stride;
    p.tnext = ctx->d_tnext;
    p.cursor = ctx->d_sync;
    p.ticket = ctx->d_sync + 1;
    p.prog = ctx->d_prog;
    p.inst_cost = ctx->have_cost ? ctx->d_cost : nullptr;
    round_keys(seed, p.rk0, p.rk1);
    p.budget = ctx->budget;
    p.renorm_mask = (1u << ctx->renorm_log2) - 1u;
    p.counts = (unsigned long long *)out.counts;
    p.wilson = out.wilson;
    p.z = z;
    p.o_verdict = out.verdict;
    p.o_status = out.status;
    p.o_events = out.events;
    p.o_tfinal = out.t_final;
    p.o_xfinal = out.x_final;
    p.out_base = out_base;
    p.out_stride = out_stride;
    p.x_stride = ctx->s_max;
}

// Autotuner: for each precision, times short trial launches (a fixed trial
// seed, about one trajectory per resident lane, counts into a scratch
// buffer) over warps per block {2, 4, 8} x refill threshold {1, 8} for every
// size class, then the best per-class shapes against one launch over all
// instances, and keeps the fastest.  Results do not depend on the choice
// (random numbers are keyed by trajectory, not by lane).  Synchronous: call
// outside stream capture.
// Structure of the loaded problem as far as launch shapes depend on it: the
// size classes (instances, species, reactions, table words) and the
// monitor's per-warp clock area.
std::vector<int64_t> tune_signature(const smc_ctx *ctx)
{
    std::vector<int64_t> sig{ctx->n_inst, tc_bytes_of(ctx->prog), (int64_t)ctx->classes.size(), ctx->jit_ready};
    for (const auto &c : ctx->classes) {
        sig.push_back((int64_t)c.inst.size());
        sig.push_back(c.s_max);
        sig.push_back(c.r_max);
        sig.push_back(c.blob_words);
    }
    return sig;
}

// Longest work first: each instance's expected cost of a trajectory from
// the autotuner's trial counts (events per trajectory; a trial trajectory
// that hit the trials' event budget counts 8 budgets), the lists of the size
// classes sorted by it (costliest first: the cursor hands instances out in
// list order) and the costs kept for the warps' work stealing.  Results do
// not depend on the order (random numbers are keyed by trajectory and
// instance).
int order_by_cost(smc_ctx *ctx, cudaStream_t s, uint64_t trial_budget)
{
    const int n = ctx->n_inst;
    if (n < 2) return SMC_OK;
    std::vector<unsigned long long> c((size_t)n * 4);
    CK(cudaMemcpyAsync(c.data(), ctx->d_trial, c.size() * 8, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    std::vector<float> cost(n);
    for (int m = 0; m < n; ++m) {
        const double runs = (double)(c[4 * m + 1] + c[4 * m + 3]);
        const double ev = (double)c[4 * m + 2] + 8.0 * (double)trial_budget * (double)c[4 * m + 3];
        cost[m] = (float)std::max(1.0, runs > 0 ? ev / runs : 1.0);
    }
    CK(cudaMemcpyAsync(ctx->d_cost, cost.data(), (size_t)n * 4, cudaMemcpyHostToDevice, s));
    std::vector<SizeClass *> all;
    for (auto &cl : ctx->classes) all.push_back(&cl);
    all.push_back(&ctx->single);
    for (SizeClass *cl : all) {
        std::stable_sort(cl->inst.begin(), cl->inst.end(), [&](int a, int b) { return cost[a] > cost[b]; });
        CK(cudaMemcpyAsync(cl->d_list, cl->inst.data(), cl->inst.size() * 4, cudaMemcpyHostToDevice, s));
    }
    CK(cudaStreamSynchronize(s));
    ctx->have_cost = true;
    return SMC_OK;
}

int autotune(smc_ctx *ctx, int plain, cudaStream_t s)
{
    // (the trace monitor keeps the default shape: its trials would time the
    // formula's evaluation, not the launch shape)
    if (!ctx->autotune || ctx->explicit_shape || ctx->tuned[plain] || ctx->nest_mode) return SMC_OK;
    const std::vector<int64_t> sig = tune_signature(ctx);
    auto &memo = ctx->memo[plain];
    if (memo.valid && memo.sig == sig) {
        for (size_t i = 0; i < ctx->classes.size(); ++i) ctx->classes[i].shape[plain] = memo.cls[i];
        ctx->single.shape[plain] = memo.single;
        ctx->use_single[plain] = memo.use_single;
        ctx->tuned[plain] = true;
        return SMC_OK;
    }
    const uint64_t n = (uint64_t)ctx->n_inst;
    // about four trajectories per resident lane, so that the trial sees lanes
    // being refilled (one wave would measure only its slowest trajectory)
    const uint64_t lanes = (uint64_t)ctx->n_sm * 1024 * 4;
    const uint64_t per = std::max<uint64_t>(1, (lanes + n - 1) / n);
    smc_sim_out o;
    std::memset(&o, 0, sizeof(o));
    o.counts = (uint64_t *)ctx->d_trial;
    SsaParams pc;
    fill_common(ctx, pc, 0x5EED5EED5EEDull, 0.0, o, 0, per, true);
    // trials measure the bulk throughput: a short event budget keeps a rare
    // very long trajectory from dominating every trial
    pc.budget = std::min<uint64_t>(pc.budget, 1u << 13);
    CK(cudaMemsetAsync(ctx->d_trial, 0, (size_t)n * 4 * 8, s));  // the trials' counts give the costs
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    auto time_it = [&](const SizeClass &c, const Shape &sh, float &ms) -> int {
        Launch L;
        if (plan_class(ctx, plain, c, sh, L) != SMC_OK) { ms = 1e30f; ctx->err.clear(); return SMC_OK; }
        CK(cudaEventRecord(e0, s));
        int rc = issue_class(ctx, plain, pc, L, s);
        if (rc) return rc;
        CK(cudaEventRecord(e1, s));
        CK(cudaEventSynchronize(e1));
        CK(cudaEventElapsedTime(&ms, e0, e1));
        return SMC_OK;
    };
    const int warps_c[] = {2, 4, 8}, refill_c[] = {1, 8};
    int rc = SMC_OK;
    float split_total = 0.0f, ms = 0.0f;
    for (auto &c : ctx->classes) {
        Shape best = c.shape[plain];
        float best_ms = 1e30f;
        rc = time_it(c, best, ms);  // warm-up (module load, clocks)
        for (int w : warps_c)
            for (int r : refill_c) {
                if (rc) break;
                Shape sh;
                sh.warps = w;
                sh.refill = r;
                sh.blocks_sm = 0;
                rc = time_it(c, sh, ms);
                if (ms < best_ms) { best_ms = ms; best = sh; }
            }
        best.tuned = true;
        c.shape[plain] = best;
        split_total += best_ms;
    }
    ctx->use_single[plain] = false;
    if (!rc && ctx->classes.size() > 1) {
        float best_ms = 1e30f;
        Shape best = ctx->single.shape[plain];
        for (int w : warps_c)
            for (int r : refill_c) {
                if (rc) break;
                Shape sh;
                sh.warps = w;
                sh.refill = r;
                sh.blocks_sm = 0;
                rc = time_it(ctx->single, sh, ms);
                if (ms < best_ms) { best_ms = ms; best = sh; }
            }
        best.tuned = true;
        ctx->single.shape[plain] = best;
        ctx->use_single[plain] = best_ms < split_total;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc) return rc;
    rc = order_by_cost(ctx, s, pc.budget);
    if (rc) return rc;
    ctx->tuned[plain] = true;
    memo.valid = true;
    memo.sig = sig;
    memo.cls.clear();
    for (const auto &c : ctx->classes) memo.cls.push_back(c.shape[plain]);
    memo.single = ctx->single.shape[plain];
    memo.use_single = ctx->use_single[plain];
    return SMC_OK;
}

// Launches queue initialisation and the SSA kernel for every class of the
// partition in use.  Ranges (d_tbegin, d_tend) must already be on the device.
int launch_all(smc_ctx *ctx, int plain, uint64_t seed, double z, const smc_sim_out &out,
               uint64_t out_base, uint64_t out_stride, cudaStream_t s, bool uniform)
{
    SsaParams pc;
    fill_common(ctx, pc, seed, z, out, out_base, out_stride, uniform);
    for (const SizeClass *c : active_classes(ctx, plain)) {
        Launch L;
        int rc = plan_class(ctx, plain, *c, c->shape[plain ? 1 : 0], L);
        if (rc) return rc;
        rc = issue_class(ctx, plain, pc, L, s);
        if (rc) return rc;
    }
    return SMC_OK;
}

}  // namespace

// ===========================================================================
extern "C" {

const char *smc_strerror(int code)
{
    switch (code) {
    case SMC_OK: return "ok";
    case SMC_E_INVALID_ARG: return "invalid argument";
    case SMC_E_OOM: return "out of memory";
    case SMC_E_CUDA: return "CUDA error";
    case SMC_E_UNSUPPORTED: return "unsupported formula or model size";
    case SMC_E_STATE: return "model or property not loaded";
    case SMC_E_NO_DEVICE: return "no suitable CUDA device";
    default: return "unknown error";
    }
}

const char *smc_last_error(const smc_ctx *ctx) { return ctx ? ctx->err.c_str() : ""; }

int smc_create(smc_ctx **out, int device)
{
    if (!out) return SMC_E_INVALID_ARG;
    *out = nullptr;
    int n = 0;
    if (cudaGetDeviceCount(&n) != cudaSuccess || device < 0 || device >= n) return SMC_E_NO_DEVICE;
    cudaDeviceProp prop;
    if (cudaGetDeviceProperties(&prop, device) != cudaSuccess) return SMC_E_NO_DEVICE;
    if (prop.major != 10 || prop.minor != 3) return SMC_E_NO_DEVICE;
    smc_ctx *ctx = new (std::nothrow) smc_ctx();
    if (!ctx) return SMC_E_OOM;
    ctx->device = device;
    ctx->n_sm = prop.multiProcessorCount;
    ctx->smem_optin = prop.sharedMemPerBlockOptin;
    if (cudaSetDevice(device) != cudaSuccess ||
        cudaStreamCreateWithFlags(&ctx->stream, cudaStreamNonBlocking) != cudaSuccess) {
        delete ctx;
        return SMC_E_CUDA;
    }
    std::vector<uint64_t> tab(SMC_LOGTAB_BYTES / 8, 0);
    if (fp64i_log_table(tab.data())) {
        smc_destroy(ctx);
        return SMC_E_UNSUPPORTED;
    }
    if (cudaMalloc(&ctx->d_logtab, SMC_LOGTAB_BYTES) != cudaSuccess ||
        cudaMemcpy(ctx->d_logtab, tab.data(), SMC_LOGTAB_BYTES, cudaMemcpyHostToDevice) != cudaSuccess) {
        smc_destroy(ctx);
        return SMC_E_CUDA;
    }
    *out = ctx;
    return SMC_OK;
}

void smc_destroy(smc_ctx *ctx)
{
    if (!ctx) return;
    cudaSetDevice(ctx->device);
    if (ctx->stream) cudaStreamSynchronize(ctx->stream);
    free_device(ctx);
    dfree(ctx->d_logtab);
    ctx->cv.release();
    if (ctx->stream) cudaStreamDestroy(ctx->stream);
    delete ctx;
}

int smc_log_fp64(smc_ctx *ctx, const double *u, uint64_t n, double *out, void *stream)
{
    if (!ctx) return SMC_E_INVALID_ARG;
    if (!u || !out) return fail(ctx, SMC_E_INVALID_ARG, "null array");
    CK(cudaSetDevice(ctx->device));
    cudaStream_t s = stream ? (cudaStream_t)stream : ctx->stream;
    if (smc_launch_log_batch(ctx->d_logtab, u, n, out, s)) return fail(ctx, SMC_E_CUDA, "log kernel launch failed");
    return SMC_OK;
}

int smc_div_fp64(smc_ctx *ctx, const double *num, const double *den, uint64_t n, double *out, void *stream)
{
    if (!ctx) return SMC_E_INVALID_ARG;
    if (n > 0 && (!num || !den || !out)) return fail(ctx, SMC_E_INVALID_ARG, "null array");
    CK(cudaSetDevice(ctx->device));
    cudaStream_t s = stream ? (cudaStream_t)stream : ctx->stream;
    if (smc_launch_div_batch(num, den, n, out, s)) return fail(ctx, SMC_E_CUDA, "division kernel launch failed");
    return SMC_OK;
}

static int load_common(smc_ctx *ctx, int n_inst, const int32_t *S, const int32_t *R,
                       const int32_t *reactants, const int32_t *stoich, const double *rates,
                       const int32_t *x0, bool same_network)
{
    if (!ctx) return SMC_E_INVALID_ARG;
    if (n_inst < 1 || !reactants || !stoich || !rates || !x0)
        return fail(ctx, SMC_E_INVALID_ARG, "null pointer or no instance");
    std::vector<int> Sv(n_inst), Rv(n_inst);
    std::vector<size_t> ro(n_inst), so(n_inst), rt(n_inst), xo(n_inst);
    size_t nr = 0, ns = 0, nrt = 0, nx = 0;
    for (int m = 0; m < n_inst; ++m) {
        Sv[m] = same_network ? S[0] : S[m];
        Rv[m] = same_network ? R[0] : R[m];
        if (!same_network || m == 0) {
            ro[m] = nr;
            so[m] = ns;
            int rc = validate_network(ctx, Sv[m], Rv[m], reactants + nr, stoich + ns);
            if (rc) return rc;
            nr += 2 * (size_t)Rv[m];
            ns += (size_t)Rv[m] * Sv[m];
        } else {
            ro[m] = ro[0];
            so[m] = so[0];
        }
        rt[m] = nrt;
        xo[m] = nx;
        int rc = validate_params(ctx, Sv[m], Rv[m], rates + nrt, x0 + nx);
        if (rc) return rc;
        nrt += Rv[m];
        nx += Sv[m];
    }
    ctx->n_inst = n_inst;
    ctx->S = Sv;
    ctx->R = Rv;
    ctx->reac_off = ro;
    ctx->st_off = so;
    ctx->rate_off = rt;
    ctx->x0_off = xo;
    ctx->reactants.assign(reactants, reactants + nr);
    ctx->stoich.assign(stoich, stoich + ns);
    ctx->rates.assign(rates, rates + nrt);
    ctx->x0.assign(x0, x0 + nx);
    ctx->s_max = *std::max_element(Sv.begin(), Sv.end());
    ctx->batch = !same_network;
    ctx->have_model = true;
    ctx->feat_species.clear();
    ctx->feat_rates = 1;
    ctx->feat_ref.clear();
    ctx->f_reac.clear();
    ctx->f_spec.clear();
    ctx->f_pow.clear();
    ctx->f_par.clear();
    ctx->have_prop = false;  // atoms refer to the species of the model
    ctx->dirty = true;
    return SMC_OK;
}

int smc_load_model(smc_ctx *ctx, int n_species, int n_reactions, const int32_t *reactants,
                   const int32_t *stoich, const double *rates, const int32_t *x0, int n_instances)
{
    return load_common(ctx, n_instances, &n_species, &n_reactions, reactants, stoich, rates, x0, true);
}

int smc_load_rate_factors(smc_ctx *ctx, int n_factors, const int32_t *reaction, const int32_t *species,
                          const int32_t *power, const double *params)
{
    if (!ctx) return SMC_E_INVALID_ARG;
    if (!ctx->have_model) return fail(ctx, SMC_E_STATE, "load a model first");
    if (ctx->batch) return fail(ctx, SMC_E_UNSUPPORTED, "rate-law factors need a single network");
    if (n_factors < 0 || (n_factors > 0 && (!reaction || !species || !power || !params)))
        return fail(ctx, SMC_E_INVALID_ARG, "bad factor arrays");
    const int S = ctx->S[0], R = ctx->R[0];
    std::vector<int> per(R, 0);
    for (int q = 0; q < n_factors; ++q) {
        if (reaction[q] < 0 || reaction[q] >= R || species[q] < 0 || species[q] >= S)
            return fail(ctx, SMC_E_INVALID_ARG, "factor reaction or species out of range");
        if (power[q] < 1 || power[q] > SMC_MAX_FACTOR_POWER)
            return fail(ctx, SMC_E_INVALID_ARG, "factor power must be 1..4");
        if (++per[reaction[q]] > SMC_MAX_FACTORS_PER_REACTION)
            return fail(ctx, SMC_E_INVALID_ARG, "at most 2 factors per reaction");
        const double *c = params + 4 * q;
        for (int i = 0; i < 4; ++i)
            if (!std::isfinite(c[i])) return fail(ctx, SMC_E_INVALID_ARG, "factor parameters must be finite");
        if (!(c[0] >= 0.0 && c[1] >= 0.0 && c[2] > 0.0 && c[3] >= 0.0))
            return fail(ctx, SMC_E_INVALID_ARG, "factor needs a0, a1, b1 >= 0 and b0 > 0");
    }
    ctx->f_reac.assign(reaction, reaction + n_factors);
    ctx->f_spec.assign(species, species + n_factors);
    ctx->f_pow.assign(power, power + n_factors);
    ctx->f_par.assign(params, params + 4 * (size_t)n_factors);
    ctx->dirty = true;
    return SMC_OK;
}

int smc_cme_reach(smc_ctx *ctx, int instance, int32_t cap, int64_t max_states, smc_cme_result *out)
{
    if (!ctx) return SMC_E_INVALID_ARG;
    if (!out) return fail(ctx, SMC_E_INVALID_ARG, "null result");
    if (!ctx->have_model || !ctx->have_prop) return fail(ctx, SMC_E_STATE, "load a model and a property first");
    if (instance < 0 || instance >= ctx->n_inst) return fail(ctx, SMC_E_INVALID_ARG, "instance out of range");
    if (cap < 0 || max_states < 1) return fail(ctx, SMC_E_INVALID_ARG, "bad cap or max_states");
    // the property must be one until / eventually / always anchored at 0 over
    // state formulas (time-bounded reachability)
    const MonProg &P = ctx->prog;
    if (P.n_units != 1 || P.u[0].nest != 0 || P.u[0].a != 0.0 || !std::isfinite(P.u[0].b) || P.unbounded)
        return fail(ctx, SMC_E_UNSUPPORTED, "exact solve needs one U / F / G anchored at 0 over state formulas");
    const int val_true = P.table[2], val_false = P.table[1];
    if (!((val_true == 2 && val_false == 1) || (val_true == 1 && val_false == 2)))
        return fail(ctx, SMC_E_UNSUPPORTED, "exact solve needs the unit or its negation at the top level");
    const int m = instance, S = ctx->S[m], nu = (int)ctx->used_atoms.size();
    std::vector<int32_t> coef((size_t)nu * S);
    std::vector<int64_t> lo(nu), hi(nu);
    std::vector<uint8_t> neg(nu);
    for (int b = 0; b < nu; ++b) {
        const int a = ctx->used_atoms[b];
        std::memcpy(&coef[(size_t)b * S], ctx->atom_coef.data() + ctx->coef_off[m] + (size_t)a * S, sizeof(int32_t) * S);
        const double bnd = ctx->per_instance_bound ? ctx->atom_bound[(size_t)m * ctx->n_atoms + a] : ctx->atom_bound[a];
        bool nb;
        smc::atom_threshold(ctx->atom_op[a], bnd, lo[b], hi[b], nb);
        neg[b] = nb;
    }
    smc::CmeModel M;
    M.S = S;
    M.R = ctx->R[m];
    M.reactants = ctx->reactants.data() + ctx->reac_off[m];
    M.stoich = ctx->stoich.data() + ctx->st_off[m];
    M.rates = ctx->rates.data() + ctx->rate_off[m];
    M.x0 = ctx->x0.data() + ctx->x0_off[m];
    M.n_fact = (int)ctx->f_reac.size();
    M.f_reac = ctx->f_reac.data();
    M.f_spec = ctx->f_spec.data();
    M.f_pow = ctx->f_pow.data();
    M.f_par = ctx->f_par.data();
    smc::CmePredicate pred;
    pred.n_atoms = nu;
    pred.coef = coef.data();
    pred.lo = lo.data();
    pred.hi = hi.data();
    pred.neg = neg.data();
    pred.goal = P.u[0].P;
    pred.stay = P.u[0].L;
    bool any_expr = false;
    const std::vector<smc::AtomExprView> ev = used_expr(ctx, any_expr);
    pred.expr = any_expr ? ev.data() : nullptr;
    CK(cudaSetDevice(ctx->device));
    smc::CmeResult r;
    const int rc = smc::cme_reach(M, pred, P.u[0].b, cap, max_states, r, ctx->err, ctx->stream);
    if (rc == -1) return SMC_E_INVALID_ARG;
    if (rc == -2) return SMC_E_OOM;
    if (rc == -3) return SMC_E_CUDA;
    if (rc == -4) return SMC_E_UNSUPPORTED;
    // the unit's probability, or its complement for a negated unit (G)
    out->p = val_true == 2 ? r.p : 1.0 - r.p;
    out->truncated = r.truncated;
    out->poisson_tail = r.poisson_tail;
    out->n_states = r.n_states;
    out->iterations = r.iterations;
    out->lambda_t = r.lambda_t;
    return SMC_OK;
}

int smc_set_atom_expression(smc_ctx *ctx, int atom, int op, const smc_token *lhs, int n_lhs,
                            const smc_token *rhs, int n_rhs)
{
    if (!ctx) return SMC_E_INVALID_ARG;
    if (!ctx->have_prop) return fail(ctx, SMC_E_STATE, "load a property first");
    if (atom < 0 || atom >= ctx->n_atoms) return fail(ctx, SMC_E_INVALID_ARG, "atom index out of range");
    if (op < SMC_OP_LT || op > SMC_OP_NE) return fail(ctx, SMC_E_INVALID_ARG, "unknown atom operator");
    if (!lhs || !rhs) return fail(ctx, SMC_E_INVALID_ARG, "null program");
    int s_min = ctx->S[0];
    for (int m = 0; m < ctx->n_inst; ++m) s_min = std::min(s_min, ctx->S[m]);
    int rc = smc::validate_tokens(lhs, n_lhs, s_min, ctx->err);
    if (rc) return rc;
    rc = smc::validate_tokens(rhs, n_rhs, s_min, ctx->err);
    if (rc) return rc;
    auto &e = ctx->atom_expr[atom];
    e.op = op;
    e.lhs.assign(lhs, lhs + n_lhs);
    e.rhs.assign(rhs, rhs + n_rhs);
    ctx->dirty = true;
    return SMC_OK;
}

int smc_load_model_batch(smc_ctx *ctx, int n_instances, const int32_t *n_species,
                         const int32_t *n_reactions, const int32_t *reactants, const int32_t *stoich,
                         const double *rates, const int32_t *x0)
{
    if (!ctx) return SMC_E_INVALID_ARG;
    if (!n_species || !n_reactions) return fail(ctx, SMC_E_INVALID_ARG, "null size arrays");
    return load_common(ctx, n_instances, n_species, n_reactions, reactants, stoich, rates, x0, false);
}

int smc_load_property(smc_ctx *ctx, int n_atoms, const int32_t *atom_coef, const int32_t *atom_op,
                      const double *atom_bound, int per_instance, const smc_node *nodes, int n_nodes,
                      double t_max_unbounded)
{
    if (!ctx) return SMC_E_INVALID_ARG;
    if (!ctx->have_model) return fail(ctx, SMC_E_STATE, "load a model first");
    if (n_atoms < 0 || (n_atoms > 0 && (!atom_coef || !atom_op || !atom_bound)))
        return fail(ctx, SMC_E_INVALID_ARG, "bad atom arrays");
    for (int a = 0; a < n_atoms; ++a)
        if (atom_op[a] < SMC_OP_LT || atom_op[a] > SMC_OP_NE)
            return fail(ctx, SMC_E_INVALID_ARG, "unknown atom operator");
    std::vector<smc::FNode> tree;
    int root = 0;
    int rc = smc::parse_formula(nodes, n_nodes, n_atoms, tree, root, ctx->err);
    if (rc) return rc;
    MonProg prog;
    NestProg nest;
    std::vector<int> used;
    rc = smc::compile_formula(tree, root, n_atoms, t_max_unbounded, prog, used, ctx->err);
    const bool nested = rc == SMC_E_UNSUPPORTED;  // outside the units' shapes: the trace monitor
    if (nested) {
        rc = smc::compile_nested(tree, root, n_atoms, t_max_unbounded, nest, used, ctx->err);
        if (!rc) {
            std::memset(&prog, 0, sizeof(prog));
            prog.n_atoms = (int)used.size();
        }
    }
    if (rc) return rc;
    const int n = ctx->n_inst;
    std::vector<size_t> coff(n);
    size_t total = 0;
    for (int m = 0; m < n; ++m) {
        if (ctx->batch || m == 0) { coff[m] = total; total += (size_t)n_atoms * ctx->S[m]; }
        else coff[m] = 0;
    }
    const size_t nb = per_instance ? (size_t)n * n_atoms : (size_t)n_atoms;
    for (size_t i = 0; i < nb; ++i)
        if (!std::isfinite(atom_bound[i])) return fail(ctx, SMC_E_INVALID_ARG, "atom bounds must be finite");
    ctx->prog = prog;
    ctx->nest_mode = nested;
    if (nested) ctx->nest = nest;
    ctx->used_atoms = used;
    ctx->n_atoms = n_atoms;
    ctx->per_instance_bound = per_instance != 0;
    ctx->atom_op.assign(atom_op, atom_op + n_atoms);
    ctx->atom_bound.assign(atom_bound, atom_bound + nb);
    ctx->atom_coef.assign(atom_coef, atom_coef + total);
    ctx->coef_off = coff;
    ctx->atom_expr.assign(n_atoms, smc_ctx::AtomExpr());
    ctx->have_prop = true;
    ctx->dirty = true;
    return SMC_OK;
}

int smc_monitor_kind(const smc_ctx *ctx)
{
    if (!ctx || !ctx->have_prop) return 0;
    return ctx->nest_mode ? 2 : 1;
}

int smc_set_option(smc_ctx *ctx, int option, double value)
{
    if (!ctx) return SMC_E_INVALID_ARG;
    switch (option) {
    case SMC_OPT_EVENT_BUDGET:
        if (!(value >= 1.0) || value > 4294967295.0) return fail(ctx, SMC_E_INVALID_ARG, "budget 1..2^32-1");
        ctx->budget = (uint64_t)value;
        return SMC_OK;
    case SMC_OPT_TRACE_CAP:
        if (!(value >= 16.0 && value <= 16777216.0)) return fail(ctx, SMC_E_INVALID_ARG, "trace capacity 16..2^24");
        if ((uint32_t)value != ctx->trace_cap) {
            ctx->trace_cap = (uint32_t)value;
            dfree(ctx->d_tr_t);
            dfree(ctx->d_tr_w);
            dfree(ctx->d_tr_m);
            ctx->tr_lanes = 0;
            ctx->tr_slots = 0;
        }
        return SMC_OK;
    case SMC_OPT_RENORM_LOG2:
        if (!(value >= 0.0 && value <= 24.0)) return fail(ctx, SMC_E_INVALID_ARG, "renorm log2 0..24");
        ctx->renorm_log2 = (int)value;
        return SMC_OK;
    case SMC_OPT_AUTOTUNE:
        ctx->autotune = value != 0.0;
        ctx->explicit_shape = false;
        ctx->tuned[0] = ctx->tuned[1] = false;
        ctx->memo[0].valid = ctx->memo[1].valid = false;
        return SMC_OK;
    case SMC_OPT_WARPS_PER_BLOCK:
        if (!(value >= 1.0 && value <= 8.0)) return fail(ctx, SMC_E_INVALID_ARG, "warps per block 1..8");
        ctx->warps = (int)value;
        break;
    case SMC_OPT_BLOCKS_PER_SM:
        if (!(value >= 0.0 && value <= 32.0)) return fail(ctx, SMC_E_INVALID_ARG, "blocks per SM 0..32");
        ctx->blocks_sm = (int)value;
        break;
    case SMC_OPT_REFILL:
        if (!(value >= 1.0 && value <= 32.0)) return fail(ctx, SMC_E_INVALID_ARG, "refill 1..32");
        ctx->refill = (int)value;
        break;
    case SMC_OPT_RECORD: ctx->record = value != 0.0; return SMC_OK;
    case SMC_OPT_JIT:
        ctx->jit = value != 0.0;
        ctx->dirty = true;  // re-prepare: kernels and tuned shapes change
        ctx->memo[0].valid = ctx->memo[1].valid = false;
        return SMC_OK;
    case SMC_OPT_SELECTION:
        if (!(value == 0.0 || value == 1.0 || value == 2.0)) return fail(ctx, SMC_E_INVALID_ARG, "selection 0, 1 or 2");
        ctx->selection = (int)value;
        ctx->memo[0].valid = ctx->memo[1].valid = false;  // launch shapes change with the warp slice
        return SMC_OK;
    default: return fail(ctx, SMC_E_INVALID_ARG, "unknown option");
    }
    std::vector<SizeClass *> all_classes;
    for (auto &c : ctx->classes) all_classes.push_back(&c);
    all_classes.push_back(&ctx->single);
    for (SizeClass *c : all_classes)
        for (int pl = 0; pl < 2; ++pl) {
            c->shape[pl].warps = ctx->warps;
            c->shape[pl].blocks_sm = ctx->blocks_sm;
            c->shape[pl].refill = ctx->refill;
        }
    // an explicit shape replaces the tuned one (and the split partition)
    ctx->use_single[0] = ctx->use_single[1] = false;
    ctx->explicit_shape = true;
    ctx->memo[0].valid = ctx->memo[1].valid = false;
    return SMC_OK;
}

int smc_get_launch_shape(smc_ctx *ctx, int precision, int index, int *n_launches, int *warps_per_block,
                         int *blocks_per_sm, int *refill, int *n_instances, int *specialized)
{
    if (!ctx) return SMC_E_INVALID_ARG;
    if (precision != SMC_PLAIN_FP64 && precision != SMC_MIXED) return fail(ctx, SMC_E_INVALID_ARG, "bad precision");
    if (ctx->dirty) return fail(ctx, SMC_E_STATE, "no prepared model: run an estimate or a simulation first");
    const int plain = precision == SMC_PLAIN_FP64;
    const std::vector<const SizeClass *> v = active_classes(ctx, plain);
    if (n_launches) *n_launches = (int)v.size();
    if (index < 0 || index >= (int)v.size()) return fail(ctx, SMC_E_INVALID_ARG, "launch index out of range");
    const SizeClass &c = *v[index];
    const Shape &sh = c.shape[plain];
    int per_sm = sh.blocks_sm;
    if (per_sm == 0) {  // as many as fit
        Launch L;
        int rc = plan_class(ctx, plain, c, sh, L);
        if (rc) return rc;
        per_sm = L.grid / ctx->n_sm;
    }
    if (warps_per_block) *warps_per_block = sh.warps;
    if (blocks_per_sm) *blocks_per_sm = per_sm;
    if (refill) *refill = sh.refill;
    if (n_instances) *n_instances = (int)c.inst.size();
    if (specialized) *specialized = ctx->jit_ready ? 1 : 0;
    return SMC_OK;
}

int smc_simulate(smc_ctx *ctx, int precision, uint64_t seed, uint64_t traj_begin, uint64_t n_traj,
                 double confidence, const smc_sim_out *out, void *stream)
{
    if (!ctx) return SMC_E_INVALID_ARG;
    if (!out || !out->counts) return fail(ctx, SMC_E_INVALID_ARG, "counts output required");
    if (precision != SMC_PLAIN_FP64 && precision != SMC_MIXED) return fail(ctx, SMC_E_INVALID_ARG, "bad precision");
    if (traj_begin + n_traj > (1ull << 32)) return fail(ctx, SMC_E_INVALID_ARG, "trajectory index >= 2^32");
    if (out->wilson && !(confidence > 0.0 && confidence < 1.0))
        return fail(ctx, SMC_E_INVALID_ARG, "confidence must lie in (0,1)");
    int rc = prepare(ctx);
    if (rc) return rc;
    CK(cudaSetDevice(ctx->device));
    cudaStream_t s = stream ? (cudaStream_t)stream : ctx->stream;
    rc = autotune(ctx, precision == SMC_PLAIN_FP64, s);
    if (rc) return rc;
    const double z = out->wilson ? z_of(confidence) : 0.0;
    return launch_all(ctx, precision == SMC_PLAIN_FP64, seed, z, *out, traj_begin, n_traj, s, true);
}

// smc_simulate without any device allocation: the model tables must already
// be resident (an earlier smc_simulate / smc_estimate put them there) and the
// SSA kernel's work queue, instance cursor and finish ticket live in the
// library's fixed scratch array (smc_noalloc_scratch) instead of buffers of
// the context.  Nothing here calls cudaMalloc, cudaFree or an allocating
// library routine: only attribute and occupancy queries and two launches per
// size class (queue reset, SSA kernel) on the caller's stream.
int smc_simulate_noalloc(smc_ctx *ctx, int precision, uint64_t seed, uint64_t traj_begin,
                         uint64_t n_traj, double confidence, const smc_sim_out *out, void *stream)
{
    if (!ctx) return SMC_E_INVALID_ARG;
    if (!out || !out->counts) return fail(ctx, SMC_E_INVALID_ARG, "counts output required");
    if (precision != SMC_PLAIN_FP64 && precision != SMC_MIXED) return fail(ctx, SMC_E_INVALID_ARG, "bad precision");
    if (traj_begin + n_traj > (1ull << 32)) return fail(ctx, SMC_E_INVALID_ARG, "trajectory index >= 2^32");
    if (out->wilson && !(confidence > 0.0 && confidence < 1.0))
        return fail(ctx, SMC_E_INVALID_ARG, "confidence must lie in (0,1)");
    if (!ctx->have_model || !ctx->have_prop || ctx->dirty || !ctx->d_blobs)
        return fail(ctx, SMC_E_STATE,
                    "model tables not on the device: call smc_simulate or smc_estimate once first");
    if (ctx->nest_mode)
        return fail(ctx, SMC_E_UNSUPPORTED, "smc_simulate_noalloc: the trace monitor's formulas need its buffers");
    if (ctx->n_inst > SMC_NOALLOC_MAX_INSTANCES)
        return fail(ctx, SMC_E_INVALID_ARG,
                    "smc_simulate_noalloc supports at most SMC_NOALLOC_MAX_INSTANCES (4096) instances");
    CK(cudaSetDevice(ctx->device));
    unsigned long long *queue = nullptr;
    unsigned int *sync = nullptr;
    if (smc_noalloc_scratch(ctx->device, &queue, &sync))
        return fail(ctx, SMC_E_CUDA, "cudaGetSymbolAddress of the scratch array failed");
    cudaStream_t s = stream ? (cudaStream_t)stream : ctx->stream;
    const int plain = precision == SMC_PLAIN_FP64;
    SsaParams p;
    std::memset(&p, 0, sizeof(p));
    p.blobs = ctx->d_blobs;
    p.blob_off = ctx->d_blob_off;
    p.n_inst = ctx->n_inst;
    p.uniform = 1;
    p.u_begin = traj_begin;
    p.u_end = traj_begin + n_traj;
    p.tnext = queue;
    p.cursor = sync;
    p.ticket = sync + 1;
    p.prog = ctx->d_prog;
    round_keys(seed, p.rk0, p.rk1);
    p.budget = ctx->budget;
    p.renorm_mask = (1u << ctx->renorm_log2) - 1u;
    p.counts = (unsigned long long *)out->counts;
    p.wilson = out->wilson;
    p.z = out->wilson ? z_of(confidence) : 0.0;
    p.o_verdict = out->verdict;
    p.o_status = out->status;
    p.o_events = out->events;
    p.o_tfinal = out->t_final;
    p.o_xfinal = out->x_final;
    p.out_base = traj_begin;
    p.out_stride = n_traj;
    p.x_stride = ctx->s_max;
    for (const SizeClass *c : active_classes(ctx, plain)) {
        Launch L;
        int rc = plan_class(ctx, plain, *c, c->shape[plain ? 1 : 0], L);
        if (rc) return rc;
        // queue reset (the counters, cursor and ticket in the scratch array), then the SSA kernel
        rc = issue_class(ctx, plain, p, L, s);
        if (rc) return rc;
    }
    return SMC_OK;
}

int smc_estimate(smc_ctx *ctx, double confidence, double half_width, uint64_t seed, int mode,
                 uint64_t fixed_n, smc_result *out)
{
    if (!ctx) return SMC_E_INVALID_ARG;
    if (!out) return fail(ctx, SMC_E_INVALID_ARG, "null result array");
    const int precision = mode & 15, sampling = mode & 0xF0;
    if (precision != SMC_PLAIN_FP64 && precision != SMC_MIXED) return fail(ctx, SMC_E_INVALID_ARG, "bad precision");
    if (sampling != SMC_FIXED_N && sampling != SMC_ITERATIVE && sampling != SMC_CONSERVATIVE)
        return fail(ctx, SMC_E_INVALID_ARG, "bad sampling mode");
    if (!(confidence > 0.0 && confidence < 1.0)) return fail(ctx, SMC_E_INVALID_ARG, "confidence must lie in (0,1)");
    if (sampling != SMC_FIXED_N && !(half_width > 0.0 && half_width < 0.5))
        return fail(ctx, SMC_E_INVALID_ARG, "half width must lie in (0, 0.5)");
    if (sampling == SMC_FIXED_N && (fixed_n < 1 || fixed_n >= (1ull << 32)))
        return fail(ctx, SMC_E_INVALID_ARG, "fixed_n must lie in 1..2^32-1");
    int rc = prepare(ctx);
    if (rc) return rc;
    CK(cudaSetDevice(ctx->device));
    cudaStream_t s = ctx->stream;
    const int n = ctx->n_inst;
    const double z = z_of(confidence);
    std::vector<uint64_t> n_tot(n, 0), want(n, 0);
    std::fill(want.begin(), want.end(), fig2_next(sampling, fixed_n, half_width, z, 0, 0, 0));
    const bool record = ctx->record && sampling == SMC_FIXED_N;
    if (record) {
        const uint64_t need = (uint64_t)n * fixed_n;
        if (ctx->record_n < need) {
            dfree(ctx->d_record);
            CK(cudaMalloc(&ctx->d_record, need));
            ctx->record_n = need;
        }
    }
    ctx->record_valid = 0;
    CK(cudaMemsetAsync(ctx->d_counts, 0, (size_t)n * 4 * 8, s));
    smc_sim_out o;
    std::memset(&o, 0, sizeof(o));
    o.counts = (uint64_t *)ctx->d_counts;
    o.wilson = ctx->d_wilson;
    if (record) o.verdict = ctx->d_record;
    // One Fig. 2 iteration = ranges up, queue reset + SSA kernel per class,
    // counts and interval down: captured once into a CUDA graph and replayed
    // for every iteration (the pinned range buffer is rewritten in between).
    const int plain = precision == SMC_PLAIN_FP64;
    rc = autotune(ctx, plain, s);
    if (rc) return rc;
    SsaParams pc;
    fill_common(ctx, pc, seed, z, o, 0, record ? fixed_n : 0, false);
    std::vector<Launch> plan;
    for (const SizeClass *c : active_classes(ctx, plain)) {
        Launch L;
        rc = plan_class(ctx, plain, *c, c->shape[plain], L);
        if (rc) return rc;
        plan.push_back(L);
    }
    // planning set each kernel's shared-memory limit to its last launch's
    // need; the launches run together, so each kernel gets the largest
    {
        int gen_max = 0;
        std::vector<std::pair<void *, int>> jit_max;
        for (const Launch &L : plan) {
            if (!L.kernel) {
                gen_max = std::max(gen_max, L.smem);
                continue;
            }
            bool seen = false;
            for (auto &kv : jit_max)
                if (kv.first == L.kernel) { kv.second = std::max(kv.second, L.smem); seen = true; }
            if (!seen) jit_max.emplace_back(L.kernel, L.smem);
        }
        if (gen_max && smc_ssa_set_smem_limit(plain, kvar(ctx), gen_max))
            return fail(ctx, SMC_E_CUDA, "cudaFuncSetAttribute failed");
        for (auto &kv : jit_max)
            if (smc_jit_set_smem_limit(kv.first, kv.second)) return fail(ctx, SMC_E_CUDA, "cudaFuncSetAttribute failed");
    }
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    CK(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
    {
        cudaError_t e1 = cudaMemcpyAsync(ctx->d_tbegin, ctx->h_range, n * 8, cudaMemcpyHostToDevice, s);
        cudaError_t e2 = cudaMemcpyAsync(ctx->d_tend, ctx->h_range + n, n * 8, cudaMemcpyHostToDevice, s);
        int lrc = (e1 == cudaSuccess && e2 == cudaSuccess) ? SMC_OK : SMC_E_CUDA;
        for (const Launch &L : plan)
            if (lrc == SMC_OK) lrc = issue_class(ctx, plain, pc, L, s);
        cudaError_t e3 = cudaMemcpyAsync(ctx->h_counts, ctx->d_counts, (size_t)n * 4 * 8, cudaMemcpyDeviceToHost, s);
        cudaError_t e4 = cudaMemcpyAsync(ctx->h_wilson, ctx->d_wilson, (size_t)n * 3 * 8, cudaMemcpyDeviceToHost, s);
        cudaError_t e5 = cudaStreamEndCapture(s, &graph);
        if (lrc != SMC_OK || e3 != cudaSuccess || e4 != cudaSuccess || e5 != cudaSuccess) {
            if (graph) cudaGraphDestroy(graph);
            return fail(ctx, SMC_E_CUDA, "capturing the estimate's launch sequence failed: " + ctx->err);
        }
    }
    if (cudaGraphInstantiate(&exec, graph, 0) != cudaSuccess) {
        cudaGraphDestroy(graph);
        return fail(ctx, SMC_E_CUDA, "cudaGraphInstantiate failed");
    }
    struct GraphGuard {
        cudaGraph_t g;
        cudaGraphExec_t x;
        ~GraphGuard() { cudaGraphExecDestroy(x); cudaGraphDestroy(g); }
    } guard{graph, exec};
    int iters = 0;
    for (;;) {
        ++iters;
        for (int m = 0; m < n; ++m) {
            ctx->h_range[m] = n_tot[m];
            ctx->h_range[n + m] = n_tot[m] + want[m];
            if (ctx->h_range[n + m] > (1ull << 32)) return fail(ctx, SMC_E_INVALID_ARG, "more than 2^32 trajectories");
        }
        CK(cudaGraphLaunch(exec, s));
        CK(cudaStreamSynchronize(s));
        bool more = false;
        for (int m = 0; m < n; ++m) {
            n_tot[m] += want[m];
            want[m] = fig2_next(sampling, fixed_n, half_width, z, ctx->h_counts[4 * m], ctx->h_counts[4 * m + 1],
                                n_tot[m]);
            more |= want[m] > 0;
        }
        if (!more) break;
    }
    for (int m = 0; m < n; ++m) {
        smc_result &r = out[m];
        r.yes = ctx->h_counts[4 * m];
        r.n = ctx->h_counts[4 * m + 1];
        r.events = ctx->h_counts[4 * m + 2];
        r.budget_hits = ctx->h_counts[4 * m + 3];
        r.launched = r.n + r.budget_hits;
        r.p_hat = ctx->h_wilson[3 * m];
        r.lo = ctx->h_wilson[3 * m + 1];
        r.hi = ctx->h_wilson[3 * m + 2];
        r.status = r.budget_hits ? SMC_STATUS_BUDGET : 0;
        r.iterations = iters;
    }
    if (record) ctx->record_valid = (uint64_t)n * fixed_n;
    return SMC_OK;
}

int smc_get_verdicts(smc_ctx *ctx, uint8_t *out, uint64_t n)
{
    if (!ctx) return SMC_E_INVALID_ARG;
    if (!ctx->record_valid) return fail(ctx, SMC_E_STATE, "no verdicts recorded");
    if (!out || n != ctx->record_valid) return fail(ctx, SMC_E_INVALID_ARG, "n must equal n_inst * fixed_n");
    CK(cudaMemcpy(out, ctx->d_record, n, cudaMemcpyDeviceToHost));
    return SMC_OK;
}

double smc_normal_quantile(double p) { return as241(p); }

int smc_wilson_interval(uint64_t yes, uint64_t n, double confidence, double *lo, double *hi)
{
    if (!lo || !hi || yes > n || !(confidence > 0.0 && confidence < 1.0)) return SMC_E_INVALID_ARG;
    double p;
    wilson_host(yes, n, z_of(confidence), &p, lo, hi);
    return SMC_OK;
}

double smc_wilson_sample(double p, double half_width, double confidence)
{
    if (!(confidence > 0.0 && confidence < 1.0) || !(half_width > 0.0)) return std::nan("");
    return wilson_sample_real(p, half_width, z_of(confidence));
}

int smc_fig2_next_batch(int sampling, uint64_t fixed_n, double confidence, double half_width, uint64_t yes,
                        uint64_t n, uint64_t n_tot, uint64_t *next)
{
    if (!next) return SMC_E_INVALID_ARG;
    if (sampling != SMC_FIXED_N && sampling != SMC_ITERATIVE && sampling != SMC_CONSERVATIVE)
        return SMC_E_INVALID_ARG;
    if (!(confidence > 0.0 && confidence < 1.0) || yes > n || n > n_tot) return SMC_E_INVALID_ARG;
    if (sampling == SMC_FIXED_N && (fixed_n < 1 || fixed_n >= (1ull << 32))) return SMC_E_INVALID_ARG;
    if (sampling != SMC_FIXED_N && !(half_width > 0.0 && half_width < 0.5)) return SMC_E_INVALID_ARG;
    *next = fig2_next(sampling, fixed_n, half_width, z_of(confidence), yes, n, n_tot);
    return SMC_OK;
}

// Diagnostic: replays given paths through the compiled monitor on the GPU
// (single-network models; atoms as loaded).  Host arrays: len[n_paths],
// x[sum len][S], t[sum len], tmin[n_paths], closed[n_paths]; outputs
// verdict[n_paths] (0 undetermined, 1 false, 2 true) and decided_at[n_paths].
int smc_monitor_replay(smc_ctx *ctx, int n_paths, const int32_t *len, const int32_t *x,
                       const double *t, const double *tmin, const uint8_t *closed, int32_t *verdict,
                       int64_t *decided_at)
{
    if (!ctx) return SMC_E_INVALID_ARG;
    if (!ctx->have_model || !ctx->have_prop) return fail(ctx, SMC_E_STATE, "load a model and a property first");
    if (ctx->batch) return fail(ctx, SMC_E_UNSUPPORTED, "replay needs a single network");
    {
        bool any_expr = false;
        used_expr(ctx, any_expr);
        if (any_expr) return fail(ctx, SMC_E_UNSUPPORTED, "replay supports linear atoms only");
    }
    if (n_paths < 1 || !len || !x || !t || !tmin || !closed || !verdict || !decided_at)
        return fail(ctx, SMC_E_INVALID_ARG, "bad replay arrays");
    CK(cudaSetDevice(ctx->device));
    const int S = ctx->S[0], nu = (int)ctx->used_atoms.size();
    std::vector<int64_t> off(n_paths);
    int64_t total = 0;
    for (int i = 0; i < n_paths; ++i) {
        if (len[i] < 1) return fail(ctx, SMC_E_INVALID_ARG, "empty path");
        off[i] = total;
        total += len[i];
    }
    std::vector<int32_t> coef((size_t)std::max(nu, 1) * S, 0);
    std::vector<int64_t> thr(2 * (size_t)std::max(nu, 1), 0);
    uint32_t neg = 0;
    for (int b = 0; b < nu; ++b) {
        const int a = ctx->used_atoms[b];
        std::memcpy(&coef[(size_t)b * S], ctx->atom_coef.data() + (size_t)a * S, sizeof(int32_t) * S);
        bool ng;
        smc::atom_threshold(ctx->atom_op[a], ctx->atom_bound[a], thr[2 * b], thr[2 * b + 1], ng);
        if (ng) neg |= 1u << b;
    }
    MonProg *d_prog = nullptr;
    NestProg *d_nest = nullptr;
    uint32_t *d_w = nullptr;
    int32_t *d_coef = nullptr, *d_len = nullptr, *d_x = nullptr, *d_v = nullptr;
    int64_t *d_thr = nullptr, *d_off = nullptr, *d_q = nullptr;
    double *d_t = nullptr, *d_tmin = nullptr;
    uint8_t *d_closed = nullptr;
    int rc = SMC_OK;
    auto run = [&]() -> int {
        CK(cudaMalloc(&d_prog, sizeof(MonProg)));
        CK(cudaMalloc(&d_coef, coef.size() * 4));
        CK(cudaMalloc(&d_thr, thr.size() * 8));
        CK(cudaMalloc(&d_len, n_paths * 4));
        CK(cudaMalloc(&d_off, n_paths * 8));
        CK(cudaMalloc(&d_x, (size_t)total * S * 4));
        CK(cudaMalloc(&d_t, (size_t)total * 8));
        CK(cudaMalloc(&d_tmin, n_paths * 8));
        CK(cudaMalloc(&d_closed, n_paths));
        CK(cudaMalloc(&d_v, n_paths * 4));
        CK(cudaMalloc(&d_q, n_paths * 8));
        CK(cudaMemcpy(d_prog, &ctx->prog, sizeof(MonProg), cudaMemcpyHostToDevice));
        CK(cudaMemcpy(d_coef, coef.data(), coef.size() * 4, cudaMemcpyHostToDevice));
        CK(cudaMemcpy(d_thr, thr.data(), thr.size() * 8, cudaMemcpyHostToDevice));
        CK(cudaMemcpy(d_len, len, n_paths * 4, cudaMemcpyHostToDevice));
        CK(cudaMemcpy(d_off, off.data(), n_paths * 8, cudaMemcpyHostToDevice));
        CK(cudaMemcpy(d_x, x, (size_t)total * S * 4, cudaMemcpyHostToDevice));
        CK(cudaMemcpy(d_t, t, (size_t)total * 8, cudaMemcpyHostToDevice));
        CK(cudaMemcpy(d_tmin, tmin, n_paths * 8, cudaMemcpyHostToDevice));
        CK(cudaMemcpy(d_closed, closed, n_paths, cudaMemcpyHostToDevice));
        if (ctx->nest_mode) {
            CK(cudaMalloc(&d_nest, sizeof(NestProg)));
            CK(cudaMemcpy(d_nest, &ctx->nest, sizeof(NestProg), cudaMemcpyHostToDevice));
            CK(cudaMalloc(&d_w, (size_t)total * 4));
        }
        ReplayParams rp;
        rp.prog = d_prog;
        rp.coef = d_coef;
        rp.athr = d_thr;
        rp.aneg = neg;
        rp.S = S;
        rp.n_paths = n_paths;
        rp.len = d_len;
        rp.off = d_off;
        rp.x = d_x;
        rp.t = d_t;
        rp.tmin = d_tmin;
        rp.closed = d_closed;
        rp.verdict = d_v;
        rp.decided_at = d_q;
        rp.nest = d_nest;
        rp.w = d_w;
        if (smc_launch_replay(rp, nullptr)) return fail(ctx, SMC_E_CUDA, "replay launch failed");
        CK(cudaMemcpy(verdict, d_v, n_paths * 4, cudaMemcpyDeviceToHost));
        CK(cudaMemcpy(decided_at, d_q, n_paths * 8, cudaMemcpyDeviceToHost));
        return SMC_OK;
    };
    rc = run();
    dfree(d_prog); dfree(d_coef); dfree(d_thr); dfree(d_len); dfree(d_off); dfree(d_x);
    dfree(d_t); dfree(d_tmin); dfree(d_closed); dfree(d_v); dfree(d_q); dfree(d_nest); dfree(d_w);
    return rc;
}

int smc_simulate_snapshot(smc_ctx *ctx, int precision, uint64_t seed, uint64_t traj_begin, uint64_t n_traj,
                          double t_snap, int stop_at_snap, const smc_sim_out *out, uint8_t *snap,
                          int32_t *x_snap, uint32_t *e_snap, void *stream)
{
    if (!ctx) return SMC_E_INVALID_ARG;
    if (!out || !out->counts || !out->verdict || !snap || !x_snap)
        return fail(ctx, SMC_E_INVALID_ARG, "counts, verdict, snap and x_snap outputs required");
    if (precision != SMC_PLAIN_FP64 && precision != SMC_MIXED) return fail(ctx, SMC_E_INVALID_ARG, "bad precision");
    if (traj_begin + n_traj > (1ull << 32)) return fail(ctx, SMC_E_INVALID_ARG, "trajectory index >= 2^32");
    if (!(t_snap >= 0.0) || !std::isfinite(t_snap)) return fail(ctx, SMC_E_INVALID_ARG, "t_snap must be finite, >= 0");
    if (ctx->nest_mode)
        return fail(ctx, SMC_E_UNSUPPORTED, "snapshots need the monitor's units (the formula needs the trace monitor)");
    int rc = prepare(ctx);
    if (rc) return rc;
    CK(cudaSetDevice(ctx->device));
    cudaStream_t s = stream ? (cudaStream_t)stream : ctx->stream;
    const int plain = precision == SMC_PLAIN_FP64;
    rc = autotune(ctx, plain, s);
    if (rc) return rc;
    smc_sim_out o = *out;
    o.wilson = nullptr;
    SsaParams pc;
    fill_common(ctx, pc, seed, 0.0, o, traj_begin, n_traj, true);
    pc.snap_mode = stop_at_snap ? 2 : 1;
    pc.t_snap = t_snap;
    pc.o_snap = snap;
    pc.o_xsnap = x_snap;
    pc.o_esnap = e_snap;
    for (const SizeClass *c : active_classes(ctx, plain)) {
        Launch L;
        rc = plan_class(ctx, plain, *c, c->shape[plain], L);
        if (rc) return rc;
        rc = issue_class(ctx, plain, pc, L, s);
        if (rc) return rc;
    }
    return SMC_OK;
}

// Number of snapshot features of a single-network context (see smc_set_features).
static int feature_count(const smc_ctx *ctx)
{
    const int Fs = ctx->feat_species.empty() ? ctx->S[0] : (int)ctx->feat_species.size();
    return Fs + 1 + (ctx->feat_rates ? ctx->R[0] : 0);
}

int smc_set_features(smc_ctx *ctx, const int32_t *species, int n_species, int with_rates,
                     const double *log_rate_ref)
{
    if (!ctx) return SMC_E_INVALID_ARG;
    if (!ctx->have_model) return fail(ctx, SMC_E_STATE, "load a model first");
    if (ctx->batch) return fail(ctx, SMC_E_UNSUPPORTED, "features need a single network");
    const int S = ctx->S[0], R = ctx->R[0];
    if (n_species < 0 || (n_species > 0 && !species)) return fail(ctx, SMC_E_INVALID_ARG, "bad species list");
    for (int i = 0; i < n_species; ++i)
        if (species[i] < 0 || species[i] >= S) return fail(ctx, SMC_E_INVALID_ARG, "species index out of range");
    const int F = (n_species ? n_species : S) + 1 + (with_rates ? R : 0);
    if (F > 16) return fail(ctx, SMC_E_UNSUPPORTED, "more than 16 features");
    if (with_rates && log_rate_ref)
        for (int j = 0; j < R; ++j)
            if (!std::isfinite(log_rate_ref[j])) return fail(ctx, SMC_E_INVALID_ARG, "log_rate_ref not finite");
    ctx->feat_species.assign(species, species + n_species);
    ctx->feat_rates = with_rates ? 1 : 0;
    if (with_rates && log_rate_ref) ctx->feat_ref.assign(log_rate_ref, log_rate_ref + R);
    else ctx->feat_ref.clear();
    return SMC_OK;
}

int smc_snapshot_features(smc_ctx *ctx, uint64_t n_traj, const int32_t *x_snap, double t_snap,
                          const float *x_scale, float t_scale, float *feat, void *stream)
{
    if (!ctx) return SMC_E_INVALID_ARG;
    if (!ctx->have_model) return fail(ctx, SMC_E_STATE, "load a model first");
    if (ctx->batch) return fail(ctx, SMC_E_UNSUPPORTED, "features need a single network");
    if (!x_snap || !x_scale || !feat || !(t_scale > 0.0f)) return fail(ctx, SMC_E_INVALID_ARG, "bad feature arguments");
    const int S = ctx->S[0], n = ctx->n_inst;
    const int R = ctx->feat_rates ? ctx->R[0] : 0;
    if (feature_count(ctx) > 16) return fail(ctx, SMC_E_UNSUPPORTED, "more than 16 features (see smc_set_features)");
    std::vector<int32_t> sidx(ctx->feat_species);
    if (sidx.empty())
        for (int i = 0; i < S; ++i) sidx.push_back(i);
    const int Fs = (int)sidx.size();
    for (int i = 0; i < Fs; ++i)
        if (!(x_scale[i] > 0.0f)) return fail(ctx, SMC_E_INVALID_ARG, "x_scale must be > 0");
    CK(cudaSetDevice(ctx->device));
    cudaStream_t s = stream ? (cudaStream_t)stream : ctx->stream;
    // log rate constants per instance, minus the reference (given, or their
    // mean over the instances)
    std::vector<float> aux(2 * (size_t)Fs + (size_t)n * R);
    for (int j = 0; j < R; ++j) {
        double ref = 0.0;
        if (!ctx->feat_ref.empty()) {
            ref = ctx->feat_ref[j];
        } else {
            for (int m = 0; m < n; ++m) {
                const double c = ctx->rates[ctx->rate_off[m] + j];
                ref += c > 0.0 ? std::log(c) : 0.0;
            }
            ref /= n;
        }
        for (int m = 0; m < n; ++m) {
            const double c = ctx->rates[ctx->rate_off[m] + j];
            aux[2 * (size_t)Fs + (size_t)m * R + j] = (float)((c > 0.0 ? std::log(c) : 0.0) - ref);
        }
    }
    std::memcpy(aux.data(), x_scale, Fs * sizeof(float));
    std::memcpy(aux.data() + Fs, sidx.data(), Fs * sizeof(int32_t));  // indices as their bits
    if (ctx->feat_aux_n < aux.size()) {
        dfree(ctx->d_feat_aux);
        CK(cudaMalloc(&ctx->d_feat_aux, aux.size() * sizeof(float)));
        ctx->feat_aux_n = aux.size();
    }
    CK(cudaMemcpyAsync(ctx->d_feat_aux, aux.data(), aux.size() * sizeof(float), cudaMemcpyHostToDevice, s));
    CK(cudaStreamSynchronize(s));  // aux is a host temporary
    if (smc_launch_snapshot_features((uint64_t)n * n_traj, n_traj, Fs,
                                     reinterpret_cast<const int32_t *>(ctx->d_feat_aux + Fs), R, ctx->s_max, x_snap,
                                     ctx->d_feat_aux, (float)(t_snap / t_scale), ctx->d_feat_aux + 2 * Fs, feat, s))
        return fail(ctx, SMC_E_CUDA, "feature kernel launch failed");
    return SMC_OK;
}

int smc_estimate_cv(smc_ctx *ctx, smc_mlp *mlp, double confidence, double half_width, uint64_t seed,
                    int precision, double t_snap, const float *x_scale, float t_scale, double beta,
                    uint64_t pilot, smc_cv_result *out)
{
    if (!ctx) return SMC_E_INVALID_ARG;
    if (!mlp || !out || !x_scale) return fail(ctx, SMC_E_INVALID_ARG, "null argument");
    if (!ctx->have_model || !ctx->have_prop) return fail(ctx, SMC_E_STATE, "load a model and a property first");
    if (ctx->n_inst != 1 || ctx->batch) return fail(ctx, SMC_E_UNSUPPORTED, "control variate needs one instance");
    if (ctx->nest_mode)
        return fail(ctx, SMC_E_UNSUPPORTED, "the control variate needs the monitor's units (the formula needs the trace monitor)");
    if (!(confidence > 0.0 && confidence < 1.0) || !(half_width > 0.0 && half_width < 0.5) || pilot < 2 ||
        !std::isfinite(beta))
        return fail(ctx, SMC_E_INVALID_ARG, "bad confidence, half width, pilot or beta");
    const uint64_t kPrefixBase = 1ull << 31;
    const int F = feature_count(ctx);
    if (smc_mlp_inputs(mlp) != F)
        return fail(ctx, SMC_E_INVALID_ARG, "the network's inputs differ from the snapshot features (smc_set_features)");
    const double z = z_of(confidence);
    int rc = prepare(ctx);
    if (rc) return rc;
    CK(cudaSetDevice(ctx->device));
    cudaStream_t s = ctx->stream;
    // device buffers of the context, grown on demand
    auto &b = ctx->cv;
    auto grow = [&](uint64_t n) -> int {
        if (n <= b.cap && ctx->s_max <= b.s_cap && F <= b.f_cap) return SMC_OK;
        const uint64_t c = std::max<uint64_t>(n, 2 * b.cap);
        uint64_t *counts = b.counts;
        double *sums = b.sums;
        b.counts = nullptr;
        b.sums = nullptr;
        b.release();
        b.counts = counts;
        b.sums = sums;
        CK(cudaMalloc(&b.y, c));
        CK(cudaMalloc(&b.snap, c));
        CK(cudaMalloc(&b.x, c * ctx->s_max * 4));
        CK(cudaMalloc(&b.e, c * 4));
        CK(cudaMalloc(&b.feat, c * F * 4));
        CK(cudaMalloc(&b.g, c * 4));
        b.cap = c;
        b.s_cap = ctx->s_max;
        b.f_cap = F;
        return SMC_OK;
    };
    if (!b.counts) CK(cudaMalloc(&b.counts, 2 * 4 * 8));
    if (!b.sums) CK(cudaMalloc(&b.sums, 14 * 8));
    CK(cudaMemsetAsync(b.counts, 0, 2 * 4 * 8, s));
    CK(cudaMemsetAsync(b.sums, 0, 14 * 8, s));
    // runs trajectories [lo, hi) (full or prefix-only) and accumulates their sums
    auto run = [&](uint64_t lo, uint64_t hi, bool prefix) -> int {
        if (hi <= lo) return SMC_OK;
        const uint64_t n = hi - lo;
        int r = grow(n);
        if (r) return r;
        smc_sim_out o;
        std::memset(&o, 0, sizeof(o));
        o.counts = b.counts + (prefix ? 4 : 0);
        o.verdict = b.y;
        r = smc_simulate_snapshot(ctx, precision, seed, lo, n, t_snap, prefix ? 1 : 0, &o, b.snap, b.x, b.e, s);
        if (r) return r;
        r = smc_snapshot_features(ctx, n, b.x, t_snap, x_scale, t_scale, b.feat, s);
        if (r) return r;
        if (smc_mlp_predict_masked(mlp, b.feat, n, b.snap, b.g, s) != SMC_OK)
            return fail(ctx, SMC_E_CUDA, std::string("surrogate prediction: ") + smc_mlp_last_error(mlp));
        if (smc_launch_cv_sums(n, b.y, b.snap, b.g, b.e, prefix ? 1 : 0, b.sums + (prefix ? 7 : 0), s))
            return fail(ctx, SMC_E_CUDA, "cv sums launch failed");
        return SMC_OK;
    };
    // pilot: full runs only, at least Fig. 2's first batch (W_s at p = 1);
    // they also measure what a prefix run would cost.  Every iteration pays
    // the latency of its longest trajectory, so the loop jumps to the
    // cost-optimal sizes rather than creeping towards them.
    uint64_t n1 = 0, n2 = 0, want1 = std::max<uint64_t>(pilot, wilson_sample_n(1.0, half_width, z)), want2 = 0;
    double hs[14];
    uint64_t hc[8];
    int iters = 0;
    double p = 0.0, V = 0.0, neff = 0.0;
    for (;;) {
        ++iters;
        if (want1 >= kPrefixBase || want2 >= kPrefixBase) return fail(ctx, SMC_E_INVALID_ARG, "sample sizes exceed 2^31");
        rc = run(n1, want1, false);
        if (rc) return rc;
        rc = run(kPrefixBase + n2, kPrefixBase + want2, true);
        if (rc) return rc;
        n1 = want1;
        n2 = want2;
        CK(cudaMemcpyAsync(hs, b.sums, sizeof(hs), cudaMemcpyDeviceToHost, s));
        CK(cudaMemcpyAsync(hc, b.counts, sizeof(hc), cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        // S1: full runs (Y, G); S2: prefix runs (G only)
        for (double v : hs)
            if (!std::isfinite(v))
                return fail(ctx, SMC_E_CUDA, std::string("surrogate prediction gave non-finite values: ") +
                                                 smc_mlp_last_error(mlp));
        const double c1n = hs[0], sY = hs[1], sG1 = hs[2], sYY = hs[3], sGG1 = hs[4], sYG = hs[5];
        const double sE1 = hs[6];  // events the full runs spent up to the snapshot (or their verdict)
        const double c2n = hs[7], sG2 = hs[9], sGG2 = hs[11];
        const double nn = c1n + c2n;
        const double mD = (sY - beta * sG1) / c1n, mG1 = sG1 / c1n, mG = (sG1 + sG2) / nn;
        p = mD + beta * mG;
        const double sDD = sYY - 2.0 * beta * sYG + beta * beta * sGG1, sDG = sYG - beta * sGG1;
        const double vD = std::max(0.0, (sDD - c1n * mD * mD) / (c1n - 1.0));
        const double vG = std::max(0.0, (sGG1 + sGG2 - nn * mG * mG) / (nn - 1.0));
        const double cDG = (sDG - c1n * mD * mG1) / (c1n - 1.0);
        const double a = vD, bb = std::max(0.0, beta * beta * vG + 2.0 * beta * cDG);
        V = a / c1n + bb / nn;
        // Until the full runs hold both verdicts, the sample variance says
        // nothing about Y (the control variate only adds noise around a
        // constant): n_eff = the full runs, as Fig. 2 treats p = 0 or 1.
        const bool interior = p > 0.0 && p < 1.0 && V > 0.0 && sY > 0.0 && sY < c1n;
        neff = interior ? p * (1.0 - p) / V : c1n;
        const double pp = p <= 0.5 ? p + half_width : p - half_width;
        const double target = wilson_sample_real(pp, half_width, z);
        if (neff >= target || iters >= 64) break;
        // cost-optimal sizes for the target variance (events per run measured)
        const double c_full = std::max(1.0, (double)hc[2] / c1n), c_pre = std::max(1.0, sE1 / c1n);
        const double dcost = std::max(c_full - c_pre, 1e-3 * c_full);
        // sizes aimed 5% above the target, so that the estimates' drift
        // between iterations rarely costs another (latency-bound) iteration
        const double aim = 1.05 * target;
        uint64_t t1, t2;
        if (!interior) {  // no variance information yet: grow the full sample as Fig. 2 does
            t1 = (uint64_t)std::ceil(target);
            t2 = n2;
        } else {
            const double Vt = p * (1.0 - p) / aim;
            const double k = std::sqrt(a * dcost) + std::sqrt(bb * c_pre);
            double o1 = std::sqrt(a / dcost) * k / Vt, on = bb > 0.0 ? std::sqrt(bb / c_pre) * k / Vt : 0.0;
            if (on < o1) { o1 = (a + bb) / Vt; on = o1; }
            t1 = (uint64_t)std::ceil(o1);
            t2 = (uint64_t)std::ceil(std::max(0.0, on - o1));
        }
        // at most 1024x per iteration (a guard against a wild early estimate;
        // the pilot is already Fig. 2's first batch)
        want1 = std::min(std::max(t1, n1 + 1), 1024 * n1);
        want2 = std::min(std::max(t2, n2), 1024 * std::max(n2, n1));
    }
    out->p_hat = p;
    out->var = V;
    out->n_eff = neff;
    out->beta = beta;
    // Eq. 4 at the effective sample size
    const double dn = std::max(neff, 1.0), z2 = z * z, pc = std::min(1.0, std::max(0.0, p));
    const double centre = pc + z2 / (2.0 * dn);
    const double half = z * std::sqrt(pc * (1.0 - pc) / dn + z2 / (4.0 * dn * dn));
    const double den = 1.0 + z2 / dn;
    out->lo = std::max(0.0, (centre - half) / den);
    out->hi = std::min(1.0, (centre + half) / den);
    out->n_full = n1;
    out->n_prefix = n2;
    out->events_full = hc[2];
    out->events_prefix = hc[6];
    out->iterations = iters;
    out->status = (hc[3] || hc[7]) ? SMC_STATUS_BUDGET : 0;
    return SMC_OK;
}

}  // extern "C"
