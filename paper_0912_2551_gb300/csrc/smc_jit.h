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

namespace smc {

#define SMC_JIT_MAX_S 8
#define SMC_JIT_MAX_R 8

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
};

// The generated header for M, or "" (with the reason in why) when M is not
// eligible.
std::string jit_model_header(const JitModel &M, std::string &why);

// Kernel handles (cudaKernel_t) of the plain and mixed specialized kernels.
struct JitKernels {
    void *plain = nullptr;
    void *mixed = nullptr;
};

// Compiles (or finds in the cache) the kernels for a generated header.
// Returns 0, or -1 with the reason in err (NVRTC missing, compile or load
// failure).
int jit_compile(const std::string &model_header, JitKernels &out, std::string &err);

}  // namespace smc
