// smc_cme.h -- exact time-bounded reachability by uniformisation (see
// smc_cme.cu): the validator behind smc_cme_reach.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "smc_compile.h"

namespace smc {

// One network instance (host arrays), with optional rate-law factors.
struct CmeModel {
    int S = 0, R = 0;
    const int32_t *reactants = nullptr;  // [R][2]
    const int32_t *stoich = nullptr;     // [R][S]
    const double *rates = nullptr;       // [R]
    const int32_t *x0 = nullptr;         // [S]
    int n_fact = 0;
    const int32_t *f_reac = nullptr, *f_spec = nullptr, *f_pow = nullptr;
    const double *f_par = nullptr;
};

// State predicates over the atom bit vector (truth tables as in MonUnit):
// goal = the unit's right operand, stay = its left operand.
struct CmePredicate {
    int n_atoms = 0;
    const int32_t *coef = nullptr;  // [n_atoms][S]
    const int64_t *lo = nullptr, *hi = nullptr;
    const uint8_t *neg = nullptr;
    uint64_t goal = 0, stay = ~0ull;
    const AtomExprView *expr = nullptr;  // [n_atoms] arithmetic atoms, or null
};

struct CmeResult {
    double p = 0.0;            // P(goal reached within [0, t_end] through stay states)
    double truncated = 0.0;    // mass absorbed in states beyond the cap by t_end
    double poisson_tail = 0.0; // Poisson weight mass left out
    int64_t n_states = 0, iterations = 0;
    double lambda_t = 0.0;     // uniformisation rate x t_end
};

// Propensity of reaction k at x (FP64, mass action times rate-law factors).
double cme_propensity(const CmeModel &M, int k, const int32_t *x);

// Returns 0, or -1 (invalid model), -2 (out of memory), -3 (CUDA),
// -4 (more than max_states reachable states), with the reason in err.
int cme_reach(const CmeModel &M, const CmePredicate &pred, double t_end, int32_t cap, int64_t max_states,
              CmeResult &out, std::string &err, cudaStream_t s);

}  // namespace smc
