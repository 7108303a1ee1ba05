// smc_compile.h -- host-side formula compiler and model-table builder.
#pragma once
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/smc.h"
#include "smc_internal.h"
#include "smc_nest.h"

namespace smc {

struct FNode {
    int kind = 0, arg = -1;
    double lo = 0.0, hi = 0.0;
    int c0 = -1, c1 = -1;
};

// One instance's network, pointing into the context's host copies.
struct InstanceModel {
    int S = 0, R = 0;
    const int32_t *reactants = nullptr;  // [R][2]
    const int32_t *stoich = nullptr;     // [R][S]
    const double *rates = nullptr;       // [R]
    const int32_t *x0 = nullptr;         // [S]
    // rate-law factors (may be empty): reaction, species, power, params [4]
    int n_fact = 0;
    const int32_t *f_reac = nullptr, *f_spec = nullptr, *f_pow = nullptr;
    const double *f_par = nullptr;
};

int parse_formula(const smc_node *nodes, int n_nodes, int n_atoms, std::vector<FNode> &tree,
                  int &root, std::string &err);

// Compiles the formula tree into `prog`; used_atoms[bit] = original atom index.
int compile_formula(const std::vector<FNode> &tree, int root, int n_atoms, double t_max,
                    MonProg &prog, std::vector<int> &used_atoms, std::string &err);

// The trace monitor's program for any formula (smc_nest.h): used when
// compile_formula rejects the shape.  SMC_E_UNSUPPORTED beyond 32 nodes, a
// tree deeper than 10 or more than 6 atoms; SMC_E_INVALID_ARG for an
// interval without 0 <= lo <= hi (lo finite) or an unbounded formula
// without a finite t_max > 0.
int compile_nested(const std::vector<FNode> &tree, int root, int n_atoms, double t_max, NestProg &np,
                   std::vector<int> &used_atoms, std::string &err);

// atom  L <op> b  (L an integer)  as  lo <= L <= hi, negated when neg.
void atom_threshold(int op, double b, int64_t &lo, int64_t &hi, bool &neg);

// An arithmetic atom lhs <op> rhs (smc_set_atom_expression); op < 0: none.
struct AtomExprView {
    int op = -1;
    const smc_token *lhs = nullptr, *rhs = nullptr;
    int n_lhs = 0, n_rhs = 0;
};

// Checks a postfix program: known tokens, species < S, exponents 0..16,
// stack never empty when popped, at most SMC_EXPR_MAX_DEPTH deep, one value
// left.  0 or SMC_E_INVALID_ARG with the reason in err.
int validate_tokens(const smc_token *t, int n, int S, std::string &err);

// Evaluates a program on a state (FP64, each operation rounded once).
double eval_tokens(const smc_token *t, int n, const int32_t *x);

// lhs <op> rhs on a state.
bool expr_atom_holds(const AtomExprView &e, const int32_t *x);

// Builds the shared-memory table of one instance (layout: BlobHdr).
// expr_used (may be null): the arithmetic atoms among the used ones.
int build_blob(const InstanceModel &M, int n_used, const int32_t *coef_used, const int32_t *op_used,
               const double *bound_used, const AtomExprView *expr_used, std::vector<uint32_t> &blob,
               std::string &err);

}  // namespace smc
