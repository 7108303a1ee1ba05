// smc_jit.cpp -- code generation, run-time compilation (NVRTC) and launch of
// the model-specialized SSA kernels (smc_jit_kernel.cuh).
#include "smc_jit.h"

#include <cuda_runtime.h>
#include <dlfcn.h>
#include <nvrtc.h>

#include <cstdio>
#include <cstdlib>
#include <limits>
#include <map>
#include <mutex>
#include <sstream>
#include <type_traits>
#include <vector>

#include "smc_internal.h"
#include "smc_jit_sources.inc"  // kJitHeaderNames / kJitHeaderSources, written by build.py

namespace smc {
namespace {

// NVRTC entry points, resolved with dlopen so that the library loads (and
// the generic kernels run) on a machine without it.
struct Nvrtc {
    bool ok = false;
    std::string why;
    decltype(&nvrtcCreateProgram) create = nullptr;
    decltype(&nvrtcCompileProgram) compile = nullptr;
    decltype(&nvrtcGetProgramLogSize) log_size = nullptr;
    decltype(&nvrtcGetProgramLog) log = nullptr;
    decltype(&nvrtcGetCUBINSize) cubin_size = nullptr;
    decltype(&nvrtcGetCUBIN) cubin = nullptr;
    decltype(&nvrtcDestroyProgram) destroy = nullptr;
    decltype(&nvrtcGetErrorString) error_string = nullptr;
};

Nvrtc &nvrtc()
{
    static Nvrtc api;
    static std::once_flag once;
    std::call_once(once, [] {
        std::vector<std::string> names = {"libnvrtc.so.13", "libnvrtc.so"};
        for (const char *env : {"CUDA_HOME", "CUDA_PATH"})
            if (const char *h = std::getenv(env)) names.push_back(std::string(h) + "/lib64/libnvrtc.so.13");
        names.push_back("/usr/local/cuda/lib64/libnvrtc.so.13");
        void *h = nullptr;
        for (const auto &n : names)
            if ((h = dlopen(n.c_str(), RTLD_NOW | RTLD_LOCAL))) break;
        if (!h) { api.why = "NVRTC (libnvrtc.so.13) not found"; return; }
        auto sym = [&](auto &fn, const char *name) {
            fn = reinterpret_cast<std::remove_reference_t<decltype(fn)>>(dlsym(h, name));
            return fn != nullptr;
        };
        api.ok = sym(api.create, "nvrtcCreateProgram") && sym(api.compile, "nvrtcCompileProgram") &&
                 sym(api.log_size, "nvrtcGetProgramLogSize") && sym(api.log, "nvrtcGetProgramLog") &&
                 sym(api.cubin_size, "nvrtcGetCUBINSize") && sym(api.cubin, "nvrtcGetCUBIN") &&
                 sym(api.destroy, "nvrtcDestroyProgram") && sym(api.error_string, "nvrtcGetErrorString");
        if (!api.ok) api.why = "NVRTC is missing an entry point";
    });
    return api;
}

std::mutex g_cache_mu;
std::map<std::string, JitKernels> g_cache;  // generated header -> kernels (never unloaded)

}  // namespace

namespace {
// exact hexadecimal literals (C++17)
std::string hex_double(double v)
{
    char b[64];
    std::snprintf(b, sizeof(b), "%a", v);
    return b;
}
std::string hex_float(double v)
{
    char b[64];
    std::snprintf(b, sizeof(b), "%af", (double)(float)v);
    return b;
}
}  // namespace

void jit_layout(const JitModel &M, int &delta_bytes, int &rate_count)
{
    const bool medium = M.S > SMC_JIT_SMALL || M.R > SMC_JIT_SMALL;
    delta_bytes = medium ? (M.R * ((M.S + 3) / 4) * 4 + 15) / 16 * 16 : 0;
    rate_count = medium ? M.R : 0;
}

std::string jit_model_header(const JitModel &M, std::string &why)
{
    const int S = M.S, R = M.R;
    if (S < 1 || S > SMC_JIT_MAX_S || R < 1 || R > SMC_JIT_MAX_R) {
        why = "network larger than the specialized kernels' limit";
        return "";
    }
    const bool medium = S > SMC_JIT_SMALL || R > SMC_JIT_SMALL;
    for (int k = 0; medium && k < R; ++k)
        for (int i = 0; i < S; ++i) {
            const int32_t v = M.stoich[(size_t)k * S + i];
            if (v > 127 || v < -127) {
                why = "net change outside the specialized kernels' int8 table";
                return "";
            }
        }
    std::ostringstream o;
    o << "// generated: one network structure as code (see smc_jit_kernel.cuh)\n#pragma once\n";
    o << "#define JS " << S << "\n#define JR " << R << "\n#define JNA " << M.n_atoms << "\n";
    if (medium) {
        // net changes of reaction j as int8 bytes, (S + 3) / 4 words per row
        const int W = (S + 3) / 4;
        o << "#define JIT_MEDIUM 1\n#define JW " << W << "\n";
        o << "__device__ const uint32_t kJitDelta[" << R * W << "] = {";
        for (int k = 0; k < R; ++k)
            for (int w = 0; w < W; ++w) {
                uint32_t word = 0;
                for (int b = 0; b < 4; ++b) {
                    const int i = 4 * w + b;
                    if (i < S) word |= (uint32_t)(uint8_t)(int8_t)M.stoich[(size_t)k * S + i] << (8 * b);
                }
                o << (k || w ? ", " : "") << word << "u";
            }
        o << "};\n";
        o << "__device__ __forceinline__ void jit_apply_row(const uint32_t *row, int32_t *x, int sgn)\n{\n";
        for (int i = 0; i < S; ++i) {
            bool any = false;
            for (int k = 0; k < R; ++k) any = any || M.stoich[(size_t)k * S + i] != 0;
            if (any)
                o << "    x[" << i << "] += sgn * (int32_t)(int8_t)(row[" << i / 4 << "] >> " << 8 * (i % 4) << ");\n";
        }
        o << "}\n";
    }
    // propensities, both precisions, in the generic kernel's arithmetic
    for (int plain = 1; plain >= 0; --plain) {
        const char *T = plain ? "double" : "float";
        o << "__device__ __forceinline__ void jit_props_" << (plain ? "plain" : "mixed")
          << "(const int32_t *x, const " << T << " *c, " << T << " *pre, uint32_t &pos)\n{\n    " << T
          << " acc, a;\n";
        for (int k = 0; k < R; ++k) {
            int ra = M.reactants[2 * k], rb = M.reactants[2 * k + 1];
            if (ra < 0 && rb >= 0) { ra = rb; rb = -1; }
            std::ostringstream h;
            if (ra < 0) {
                o << "    a = c[" << k << "];\n";  // zeroth order: h = 1
            } else {
                if (plain) {
                    if (rb < 0) h << "(long long)x[" << ra << "]";
                    else if (ra != rb) h << "(long long)x[" << ra << "] * (long long)x[" << rb << "]";
                    else h << "((long long)x[" << ra << "] * (long long)(x[" << ra << "] - 1)) >> 1";
                    o << "    a = __dmul_rn(c[" << k << "], int_to_double(" << h.str() << "));\n";
                } else {
                    if (rb < 0) h << "(float)x[" << ra << "]";
                    else if (ra != rb) h << "__fmul_rn((float)x[" << ra << "], (float)x[" << rb << "])";
                    else h << "__fmul_rn((float)x[" << ra << "], __fmaf_rn((float)x[" << ra << "], 0.5f, -0.5f))";
                    o << "    a = __fmul_rn(c[" << k << "], " << h.str() << ");\n";
                }
            }
            // rate-law factors of reaction k, in order, as in the generic kernel
            for (int q = 0; q < M.n_fact; ++q) {
                if (M.f_reac[q] != k) continue;
                const double *c = M.f_par + 4 * q;
                const int m = M.f_spec[q];
                if (plain) {
                    o << "    { const double xv = int_to_double((long long)x[" << m << "]); double xn = xv;";
                    for (int i = 1; i < M.f_pow[q]; ++i) o << " xn = __dmul_rn(xn, xv);";
                    o << "\n      a = __dmul_rn(a, __ddiv_rn(__dadd_rn(" << hex_double(c[0]) << ", __dmul_rn("
                      << hex_double(c[1]) << ", xn)), __dadd_rn(" << hex_double(c[2]) << ", __dmul_rn("
                      << hex_double(c[3]) << ", xn)))); }\n";
                } else {
                    o << "    { const float xv = (float)x[" << m << "]; float xn = xv;";
                    for (int i = 1; i < M.f_pow[q]; ++i) o << " xn = __fmul_rn(xn, xv);";
                    o << "\n      a = __fmul_rn(a, __fdiv_rn(__fadd_rn(" << hex_float(c[0]) << ", __fmul_rn("
                      << hex_float(c[1]) << ", xn)), __fadd_rn(" << hex_float(c[2]) << ", __fmul_rn("
                      << hex_float(c[3]) << ", xn)))); }\n";
                }
            }
            o << "    pos |= (uint32_t)(" << (plain ? "__double_as_longlong(a) > 0" : "a > 0.0f") << ") << " << k
              << ";\n";
            if (k == 0) o << "    acc = a;\n";
            else o << "    acc = " << (plain ? "__dadd_rn" : "__fadd_rn") << "(acc, a);\n";
            o << "    pre[" << k << "] = acc;\n";
        }
        o << "}\n";
    }
    // x += v_j as selects (no divergent branch on j); medium networks use the
    // table above instead
    o << "__device__ __forceinline__ void jit_apply(int j, int32_t *x, int sgn)\n{\n";
    if (medium) o << "    (void)j; (void)x; (void)sgn;\n";
    for (int i = 0; i < S; ++i) {
        std::ostringstream d;
        for (int k = 0; k < R; ++k) {
            const int32_t v = M.stoich[(size_t)k * S + i];
            if (v) d << (d.tellp() > 0 ? " + " : "") << "(j == " << k << " ? " << v << " : 0)";
        }
        if (d.tellp() > 0 && !medium) o << "    x[" << i << "] += sgn * (" << d.str() << ");\n";
    }
    o << "}\n";
    // atoms: (lo <= L <= hi) xor neg, L = sum coef x (exact int64)
    o << "__device__ __forceinline__ uint32_t jit_atoms(const int32_t *x)\n{\n    uint32_t ab = 0;\n";
    const int64_t MIN64 = std::numeric_limits<int64_t>::min(), MAX64 = std::numeric_limits<int64_t>::max();
    int tmp = 0;
    for (int a = 0; a < M.n_atoms; ++a) {
        if (M.expr && M.expr[a].op >= 0) {  // arithmetic atom: one temporary per token, in program order
            const AtomExprView &e = M.expr[a];
            std::string side[2];
            for (int sd = 0; sd < 2; ++sd) {
                const smc_token *t = sd ? e.rhs : e.lhs;
                const int n = sd ? e.n_rhs : e.n_lhs;
                std::vector<std::string> st;
                for (int i = 0; i < n; ++i) {
                    const std::string v = "e" + std::to_string(tmp++);
                    std::string rhs;
                    switch (t[i].kind) {
                    case SMC_TOK_SPECIES: rhs = "int_to_double((long long)x[" + std::to_string(t[i].arg) + "])"; break;
                    case SMC_TOK_CONST: rhs = hex_double(t[i].value); break;
                    case SMC_TOK_SQRT: rhs = "__dsqrt_rn(" + st.back() + ")"; st.pop_back(); break;
                    case SMC_TOK_POWI: {
                        const std::string base = st.back();
                        st.pop_back();
                        if (t[i].arg == 0) rhs = "1.0";
                        else {
                            rhs = base;
                            for (int k = 1; k < t[i].arg; ++k) rhs = "__dmul_rn(" + rhs + ", " + base + ")";
                        }
                        break;
                    }
                    default: {
                        const std::string b = st.back();
                        st.pop_back();
                        const std::string x = st.back();
                        st.pop_back();
                        const char *fn = t[i].kind == SMC_TOK_ADD ? "__dadd_rn" : t[i].kind == SMC_TOK_SUB ? "__dsub_rn"
                                       : t[i].kind == SMC_TOK_MUL ? "__dmul_rn" : "__ddiv_rn";
                        rhs = std::string(fn) + "(" + x + ", " + b + ")";
                    }
                    }
                    o << "    const double " << v << " = " << rhs << ";\n";
                    st.push_back(v);
                }
                side[sd] = st.back();
            }
            static const char *cmp[] = {"<", "<=", ">=", ">", "==", "!="};
            o << "    ab |= ((uint32_t)(" << side[0] << " " << cmp[e.op] << " " << side[1] << ")) << " << a << ";\n";
            continue;
        }
        std::ostringstream L;
        int nterm = 0, single = -1;
        for (int i = 0; i < S; ++i) {
            const int32_t c = M.coef[(size_t)a * S + i];
            if (!c) continue;
            ++nterm;
            single = (c == 1) ? i : -2;
            L << (L.tellp() > 0 ? " + " : "") << "(long long)x[" << i << "]";
            if (c != 1) L << " * " << c << "LL";
        }
        const int64_t lo = M.lo[a], hi = M.hi[a];
        std::ostringstream cond;
        if (lo > hi) cond << "false";
        else if (nterm == 0) cond << ((lo <= 0 && 0 <= hi) ? "true" : "false");
        else if (nterm == 1 && single >= 0) {  // L = x_i, an int32: compare in 32 bits
            const int64_t I32MIN = std::numeric_limits<int32_t>::min(), I32MAX = std::numeric_limits<int32_t>::max();
            if (lo > I32MAX || hi < I32MIN) cond << "false";
            else {
                std::vector<std::string> parts;
                if (lo > I32MIN) parts.push_back("x[" + std::to_string(single) + "] >= " + std::to_string(lo));
                if (hi < I32MAX) parts.push_back("x[" + std::to_string(single) + "] <= " + std::to_string(hi));
                if (parts.empty()) cond << "true";
                else cond << parts[0] << (parts.size() > 1 ? " && " + parts[1] : "");
            }
        } else {
            std::vector<std::string> parts;
            if (lo != MIN64) parts.push_back("(" + L.str() + ") >= " + std::to_string(lo) + "LL");
            if (hi != MAX64) parts.push_back("(" + L.str() + ") <= " + std::to_string(hi) + "LL");
            if (parts.empty()) cond << "true";
            else cond << parts[0] << (parts.size() > 1 ? " && " + parts[1] : "");
        }
        o << "    ab |= ((uint32_t)(" << cond.str() << ")" << (M.neg[a] ? " ^ 1u" : "") << ") << " << a << ";\n";
    }
    o << "    return ab;\n}\n";
    return o.str();
}

int jit_compile(const std::string &model_header, JitKernels &out, std::string &err)
{
    std::lock_guard<std::mutex> lk(g_cache_mu);
    auto it = g_cache.find(model_header);
    if (it != g_cache.end()) {
        out = it->second;
        return 0;
    }
    Nvrtc &api = nvrtc();
    if (!api.ok) { err = api.why; return -1; }
    std::vector<const char *> names, srcs;
    for (size_t i = 0; i < sizeof(kJitHeaderNames) / sizeof(kJitHeaderNames[0]); ++i) {
        names.push_back(kJitHeaderNames[i]);
        srcs.push_back(kJitHeaderSources[i]);
    }
    names.push_back("smc_jit_model.h");
    srcs.push_back(model_header.c_str());
    nvrtcProgram prog;
    nvrtcResult r = api.create(&prog, "#include \"smc_jit_kernel.cuh\"\n", "smc_jit.cu", (int)names.size(),
                               srcs.data(), names.data());
    if (r != NVRTC_SUCCESS) { err = std::string("nvrtcCreateProgram: ") + api.error_string(r); return -1; }
    const char *opts[] = {"--gpu-architecture=sm_103a", "-std=c++17", "-lineinfo", "--fmad=true"};
    r = api.compile(prog, (int)(sizeof(opts) / sizeof(opts[0])), opts);
    if (r != NVRTC_SUCCESS) {
        size_t n = 0;
        api.log_size(prog, &n);
        std::string log(n, '\0');
        if (n) api.log(prog, &log[0]);
        api.destroy(&prog);
        err = std::string("NVRTC compile failed: ") + log.substr(0, 2000);
        return -1;
    }
    size_t n = 0;
    api.cubin_size(prog, &n);
    std::vector<char> cubin(n);
    api.cubin(prog, cubin.data());
    api.destroy(&prog);
    cudaLibrary_t lib = nullptr;
    cudaError_t e = cudaLibraryLoadData(&lib, cubin.data(), nullptr, nullptr, 0, nullptr, nullptr, 0);
    if (e != cudaSuccess) { err = std::string("cudaLibraryLoadData: ") + cudaGetErrorString(e); return -1; }
    cudaKernel_t kp = nullptr, km = nullptr;
    if ((e = cudaLibraryGetKernel(&kp, lib, "smc_jit_ssa_plain")) != cudaSuccess ||
        (e = cudaLibraryGetKernel(&km, lib, "smc_jit_ssa_mixed")) != cudaSuccess) {
        err = std::string("cudaLibraryGetKernel: ") + cudaGetErrorString(e);
        return -1;
    }
    JitKernels k;
    k.plain = (void *)kp;
    k.mixed = (void *)km;
    g_cache[model_header] = k;
    out = k;
    return 0;
}

}  // namespace smc

// launch helpers for the specialized kernels (same contract as the generic
// ones in smc_kernels.cu)
static int to_code(cudaError_t e) { return e == cudaSuccess ? 0 : -3; }

int smc_jit_set_smem_limit(void *kernel, int smem_bytes)
{
    return to_code(cudaFuncSetAttribute((const void *)kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_bytes));
}

int smc_jit_max_blocks_per_sm(void *kernel, int block, int smem_bytes, int *out)
{
    return to_code(cudaOccupancyMaxActiveBlocksPerMultiprocessor(out, (const void *)kernel, block, smem_bytes));
}

int smc_jit_launch(void *kernel, const SsaParams &p, int grid, int block, int smem_bytes, void *stream)
{
    SsaParams copy = p;
    void *args[] = {&copy};
    return to_code(cudaLaunchKernel((const void *)kernel, dim3(grid), dim3(block), args, (size_t)smem_bytes,
                                    (cudaStream_t)stream));
}
