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

    // property
    bool have_prop = false;
    MonProg prog;
    std::vector<int> used_atoms;
    int n_atoms = 0;
    bool per_instance_bound = false;
    std::vector<int32_t> atom_op;
    std::vector<double> atom_bound;   // [n_atoms] or [n_inst][n_atoms]
    std::vector<int32_t> atom_coef;   // concatenated per instance [n_atoms][S_m]
    std::vector<size_t> coef_off;

    // device state
    bool dirty = true;
    uint32_t *d_blobs = nullptr;
    uint64_t *d_blob_off = nullptr;
    MonProg *d_prog = nullptr;
    std::vector<SizeClass> classes;
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

    // options
    uint64_t budget = 1ull << 24;
    int renorm_log2 = 8;
    int autotune = 1;
    int warps = 4;
    int blocks_sm = 0;
    int refill = 1;
    int record = 0;
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
    for (auto &c : ctx->classes) dfree(c.d_list);
    ctx->classes.clear();
    dfree(ctx->d_tbegin);
    dfree(ctx->d_tend);
    dfree(ctx->d_tnext);
    dfree(ctx->d_sync);
    dfree(ctx->d_counts);
    dfree(ctx->d_wilson);
    dfree(ctx->d_record);
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
        int rc = smc::build_blob(M, nu, coef.data(), op.data(), bnd.data(), blob, ctx->err);
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
    CK(cudaMalloc(&ctx->d_blobs, all.size() * 4));
    CK(cudaMemcpy(ctx->d_blobs, all.data(), all.size() * 4, cudaMemcpyHostToDevice));
    CK(cudaMalloc(&ctx->d_blob_off, n * 8));
    CK(cudaMemcpy(ctx->d_blob_off, off.data(), n * 8, cudaMemcpyHostToDevice));
    CK(cudaMalloc(&ctx->d_prog, sizeof(MonProg)));
    CK(cudaMemcpy(ctx->d_prog, &ctx->prog, sizeof(MonProg), cudaMemcpyHostToDevice));
    for (auto &c : ctx->classes) {
        CK(cudaMalloc(&c.d_list, c.inst.size() * 4));
        CK(cudaMemcpy(c.d_list, c.inst.data(), c.inst.size() * 4, cudaMemcpyHostToDevice));
        for (int pl = 0; pl < 2; ++pl) {
            c.shape[pl].warps = ctx->warps;
            c.shape[pl].blocks_sm = ctx->blocks_sm;
            c.shape[pl].refill = ctx->refill;
        }
    }
    CK(cudaMalloc(&ctx->d_tbegin, n * 8));
    CK(cudaMalloc(&ctx->d_tend, n * 8));
    CK(cudaMalloc(&ctx->d_tnext, n * 8));
    CK(cudaMalloc(&ctx->d_sync, 16));
    CK(cudaMalloc(&ctx->d_counts, (size_t)n * 4 * 8));
    CK(cudaMalloc(&ctx->d_wilson, (size_t)n * 3 * 8));
    CK(cudaMallocHost(&ctx->h_range, (size_t)n * 2 * 8));
    CK(cudaMallocHost(&ctx->h_counts, (size_t)n * 4 * 8));
    CK(cudaMallocHost(&ctx->h_wilson, (size_t)n * 3 * 8));
    ctx->dirty = false;
    return SMC_OK;
}

// candidate clocks per warp: only formulas with a nested F / G keep them
int tc_bytes_of(const MonProg &prog)
{
    for (int u = 0; u < prog.n_units; ++u)
        if (prog.u[u].nest) return SMC_MAX_UNITS * 32 * 8;
    return 0;
}

// warp slice: table | x[(s_max + 1)][32] | tc | a[r_max][32]
int warp_bytes_of(const SizeClass &c, int plain, int tc_bytes)
{
    const int blob_words = (c.blob_words + 3) & ~3;
    const int b = blob_words * 4 + (c.s_max + 1) * 128 + tc_bytes + c.r_max * 32 * (plain ? 8 : 4);
    return (b + 15) & ~15;
}

// Launches queue initialisation and the SSA kernel for every size class.
// Ranges (d_tbegin, d_tend) must already be on the device.
int launch_all(smc_ctx *ctx, int plain, uint64_t seed, double z, const smc_sim_out &out,
               uint64_t out_base, uint64_t out_stride, cudaStream_t s, bool uniform)
{
    SsaParams p;
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
    for (auto &c : ctx->classes) {
        const Shape &sh = c.shape[plain ? 1 : 0];
        p.inst_list = c.d_list;
        p.n_list = (int)c.inst.size();
        p.refill = sh.refill;
        p.blob_words = (c.blob_words + 3) & ~3;
        p.s_max = c.s_max;
        p.r_max = c.r_max;
        p.tc_bytes = tc_bytes_of(ctx->prog);
        p.warp_bytes = warp_bytes_of(c, plain, p.tc_bytes);
        const int block = 32 * sh.warps;
        const int smem = (int)sizeof(MonProg) + sh.warps * p.warp_bytes;
        if ((size_t)smem > ctx->smem_optin)
            return fail(ctx, SMC_E_UNSUPPORTED, "model tables do not fit in shared memory");
        if (smc_ssa_set_smem_limit(plain, smem)) return fail(ctx, SMC_E_CUDA, "cudaFuncSetAttribute failed");
        int per_sm = 0;
        if (smc_ssa_max_blocks_per_sm(plain, block, smem, &per_sm) || per_sm < 1)
            return fail(ctx, SMC_E_CUDA, "occupancy query failed");
        if (sh.blocks_sm > 0) per_sm = std::min(per_sm, sh.blocks_sm);
        const int grid = ctx->n_sm * per_sm;
        if (smc_launch_queue_init(p, s)) return fail(ctx, SMC_E_CUDA, std::string("queue init: ") + cudaGetErrorString(cudaGetLastError()));
        if (smc_launch_ssa(plain, p, grid, block, smem, s))
            return fail(ctx, SMC_E_CUDA, std::string("ssa launch: ") + cudaGetErrorString(cudaGetLastError()));
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
    *out = ctx;
    return SMC_OK;
}

void smc_destroy(smc_ctx *ctx)
{
    if (!ctx) return;
    cudaSetDevice(ctx->device);
    if (ctx->stream) cudaStreamSynchronize(ctx->stream);
    free_device(ctx);
    if (ctx->stream) cudaStreamDestroy(ctx->stream);
    delete ctx;
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
    ctx->have_prop = false;  // atoms refer to the species of the model
    ctx->dirty = true;
    return SMC_OK;
}

int smc_load_model(smc_ctx *ctx, int n_species, int n_reactions, const int32_t *reactants,
                   const int32_t *stoich, const double *rates, const int32_t *x0, int n_instances)
{
    return load_common(ctx, n_instances, &n_species, &n_reactions, reactants, stoich, rates, x0, true);
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
    std::vector<int> used;
    rc = smc::compile_formula(tree, root, n_atoms, t_max_unbounded, prog, used, ctx->err);
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
    ctx->used_atoms = used;
    ctx->n_atoms = n_atoms;
    ctx->per_instance_bound = per_instance != 0;
    ctx->atom_op.assign(atom_op, atom_op + n_atoms);
    ctx->atom_bound.assign(atom_bound, atom_bound + nb);
    ctx->atom_coef.assign(atom_coef, atom_coef + total);
    ctx->coef_off = coff;
    ctx->have_prop = true;
    ctx->dirty = true;
    return SMC_OK;
}

int smc_set_option(smc_ctx *ctx, int option, double value)
{
    if (!ctx) return SMC_E_INVALID_ARG;
    switch (option) {
    case SMC_OPT_EVENT_BUDGET:
        if (!(value >= 1.0) || value > 4294967295.0) return fail(ctx, SMC_E_INVALID_ARG, "budget 1..2^32-1");
        ctx->budget = (uint64_t)value;
        return SMC_OK;
    case SMC_OPT_RENORM_LOG2:
        if (!(value >= 0.0 && value <= 24.0)) return fail(ctx, SMC_E_INVALID_ARG, "renorm log2 0..24");
        ctx->renorm_log2 = (int)value;
        return SMC_OK;
    case SMC_OPT_AUTOTUNE: ctx->autotune = value != 0.0; return SMC_OK;
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
    default: return fail(ctx, SMC_E_INVALID_ARG, "unknown option");
    }
    for (auto &c : ctx->classes)
        for (int pl = 0; pl < 2; ++pl) {
            c.shape[pl].warps = ctx->warps;
            c.shape[pl].blocks_sm = ctx->blocks_sm;
            c.shape[pl].refill = ctx->refill;
        }
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
    for (auto &c : ctx->classes) {
        const Shape &sh = c.shape[plain ? 1 : 0];
        p.inst_list = c.d_list;
        p.n_list = (int)c.inst.size();
        p.refill = sh.refill;
        p.blob_words = (c.blob_words + 3) & ~3;
        p.s_max = c.s_max;
        p.r_max = c.r_max;
        p.tc_bytes = tc_bytes_of(ctx->prog);
        p.warp_bytes = warp_bytes_of(c, plain, p.tc_bytes);
        const int block = 32 * sh.warps;
        const int smem = (int)sizeof(MonProg) + sh.warps * p.warp_bytes;
        if ((size_t)smem > ctx->smem_optin)
            return fail(ctx, SMC_E_UNSUPPORTED, "model tables do not fit in shared memory");
        if (smc_ssa_set_smem_limit(plain, smem)) return fail(ctx, SMC_E_CUDA, "cudaFuncSetAttribute failed");
        int per_sm = 0;
        if (smc_ssa_max_blocks_per_sm(plain, block, smem, &per_sm) || per_sm < 1)
            return fail(ctx, SMC_E_CUDA, "occupancy query failed");
        if (sh.blocks_sm > 0) per_sm = std::min(per_sm, sh.blocks_sm);
        // resets this launch's queue counters, cursor and ticket in the scratch array
        if (smc_launch_queue_init(p, s)) return fail(ctx, SMC_E_CUDA, "queue reset launch failed");
        if (smc_launch_ssa(plain, p, ctx->n_sm * per_sm, block, smem, s))
            return fail(ctx, SMC_E_CUDA, std::string("ssa launch: ") + cudaGetErrorString(cudaGetLastError()));
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
    uint64_t first;
    if (sampling == SMC_FIXED_N) first = fixed_n;
    else if (sampling == SMC_CONSERVATIVE) first = wilson_sample_n(0.5, half_width, z);
    else first = wilson_sample_n(1.0, half_width, z);
    std::fill(want.begin(), want.end(), first);
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
    int iters = 0;
    for (;;) {
        ++iters;
        for (int m = 0; m < n; ++m) {
            ctx->h_range[m] = n_tot[m];
            ctx->h_range[n + m] = n_tot[m] + want[m];
            if (ctx->h_range[n + m] > (1ull << 32)) return fail(ctx, SMC_E_INVALID_ARG, "more than 2^32 trajectories");
        }
        CK(cudaMemcpyAsync(ctx->d_tbegin, ctx->h_range, n * 8, cudaMemcpyHostToDevice, s));
        CK(cudaMemcpyAsync(ctx->d_tend, ctx->h_range + n, n * 8, cudaMemcpyHostToDevice, s));
        rc = launch_all(ctx, precision == SMC_PLAIN_FP64, seed, z, o, 0, record ? fixed_n : 0, s, false);
        if (rc) return rc;
        CK(cudaMemcpyAsync(ctx->h_counts, ctx->d_counts, (size_t)n * 4 * 8, cudaMemcpyDeviceToHost, s));
        CK(cudaMemcpyAsync(ctx->h_wilson, ctx->d_wilson, (size_t)n * 3 * 8, cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        bool more = false;
        for (int m = 0; m < n; ++m) {
            n_tot[m] += want[m];
            want[m] = 0;
            if (sampling != SMC_ITERATIVE) continue;
            const uint64_t yes = ctx->h_counts[4 * m], dec = ctx->h_counts[4 * m + 1];
            const double p_est = dec ? (double)yes / (double)dec : 0.0;
            const double p_prime = p_est <= 0.5 ? p_est + half_width : p_est - half_width;
            const uint64_t n_prime = wilson_sample_n(p_prime, half_width, z);
            if (n_prime > n_tot[m]) { want[m] = n_prime - n_tot[m]; more = true; }
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
        if (smc_launch_replay(rp, nullptr)) return fail(ctx, SMC_E_CUDA, "replay launch failed");
        CK(cudaMemcpy(verdict, d_v, n_paths * 4, cudaMemcpyDeviceToHost));
        CK(cudaMemcpy(decided_at, d_q, n_paths * 8, cudaMemcpyDeviceToHost));
        return SMC_OK;
    };
    rc = run();
    dfree(d_prog); dfree(d_coef); dfree(d_thr); dfree(d_len); dfree(d_off); dfree(d_x);
    dfree(d_t); dfree(d_tmin); dfree(d_closed); dfree(d_v); dfree(d_q);
    return rc;
}

}  // extern "C"
