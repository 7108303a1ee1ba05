// smc_jit.h -- model-specialized SSA kernels compiled at run time.
//
// For a network whose structure (species, reactions, reactants,
// stoichiometry, monitored atoms) is shared by every loaded instance, the
// library writes that structure as CUDA code (smc_jit_model.h), compiles the
// kernel of smc_jit_kernel.cuh with NVRTC for sm_103a and loads it with
// cudaLibraryLoadData.  Compiled kernels are cached for the life of the
// process, keyed by the generated source.  NVRTC is loaded with dlopen; when
// it is missing, or a structure is not eligible, the generic kernels run.
#pragma once
#include <stdint.h>

#include <string>

#include "smc_compile.h"

namespace smc {

#define SMC_JIT_MAX_S 32
#define SMC_JIT_MAX_R 32
// Above this size (species or reactions) the specialized kernel reads the
// fired reaction's net changes from a block-staged table and the rates from
// a per-warp shared-memory slice instead of registers.
#define SMC_JIT_SMALL 8

// One network structure with its monitored atoms (bit a of the monitor's atom
// vector = atom a here): atom a holds iff (lo_a <= sum_i coef[a][i] x_i <= hi_a)
// xor neg_a.
struct JitModel {
    int S = 0, R = 0;
    const int32_t *reactants = nullptr;  // [R][2], -1 = none
    const int32_t *stoich = nullptr;     // [R][S]
    int n_atoms = 0;
    const int32_t *coef = nullptr;       // [n_atoms][S]
    const int64_t *lo = nullptr, *hi = nullptr;
    const uint8_t *neg = nullptr;
    const AtomExprView *expr = nullptr;  // [n_atoms] arithmetic atoms, or null
    // rate-law factors (reaction, species, power, params [4]); may be empty
    int n_fact = 0;
    const int32_t *f_reac = nullptr, *f_spec = nullptr, *f_pow = nullptr;
    const double *f_par = nullptr;
};

// The generated header for M, or "" (with the reason in why) when M is not
// eligible.
std::string jit_model_header(const JitModel &M, std::string &why);

// Kernel handles (cudaKernel_t) of the plain and mixed specialized kernels,
// and the shared memory their launches add: per block, the net-change table
// (medium networks); per warp, the rates (medium networks, FP64 or FP32).
struct JitKernels {
    void *plain = nullptr;
    void *mixed = nullptr;
    int delta_bytes = 0;
    int rate_count = 0;  // R when the rates live in shared memory, else 0
};

// Shared-memory layout facts of a generated header (see jit_model_header).
void jit_layout(const JitModel &M, int &delta_bytes, int &rate_count);

// Compiles (or finds in the cache) the kernels for a generated header.
// Returns 0, or -1 with the reason in err (NVRTC missing, compile or load
// failure).
int jit_compile(const std::string &model_header, JitKernels &out, std::string &err);

}  // namespace smc
