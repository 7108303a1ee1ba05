// smc_compile.cpp -- host side: compiles a BLTLc formula (Sec. 3.1) into the
// monitor program of the SSA kernel, and builds each instance's model table.
#include "smc_compile.h"

#include <cmath>
#include <cstring>
#include <limits>

namespace smc {

namespace {

enum { V_U = 0, V_F = 1, V_T = 2 };  // unit / table value encoding

int kleene_not(int a) { return a == V_U ? V_U : (a == V_T ? V_F : V_T); }
int kleene_and(int a, int b)
{
    if (a == V_F || b == V_F) return V_F;
    if (a == V_T && b == V_T) return V_T;
    return V_U;
}
int kleene_or(int a, int b)
{
    if (a == V_T || b == V_T) return V_T;
    if (a == V_F && b == V_F) return V_F;
    return V_U;
}

bool is_temporal(int kind)
{
    return kind == SMC_NODE_UNTIL || kind == SMC_NODE_EVENTUALLY || kind == SMC_NODE_ALWAYS ||
           kind == SMC_NODE_NEXT;
}

struct Compiler {
    const std::vector<FNode> &T;
    std::vector<int> atom_bit;  // original atom index -> bit, -1 unused
    std::vector<int> used;      // bit -> original atom index
    std::string &err;

    Compiler(const std::vector<FNode> &t, std::string &e) : T(t), err(e) {}

    bool is_state(int n) const
    {
        const FNode &f = T[n];
        if (is_temporal(f.kind)) return false;
        if (f.c0 >= 0 && !is_state(f.c0)) return false;
        if (f.c1 >= 0 && !is_state(f.c1)) return false;
        return true;
    }

    bool eval_state(int n, uint32_t bits) const
    {
        const FNode &f = T[n];
        switch (f.kind) {
        case SMC_NODE_TRUE: return true;
        case SMC_NODE_FALSE: return false;
        case SMC_NODE_ATOM: return (bits >> atom_bit[f.arg]) & 1u;
        case SMC_NODE_NOT: return !eval_state(f.c0, bits);
        case SMC_NODE_AND: return eval_state(f.c0, bits) && eval_state(f.c1, bits);
        case SMC_NODE_OR: return eval_state(f.c0, bits) || eval_state(f.c1, bits);
        case SMC_NODE_IMPLIES: return !eval_state(f.c0, bits) || eval_state(f.c1, bits);
        default: return false;
        }
    }

    uint64_t table_of(int n, bool neg) const
    {
        uint64_t tt = 0;
        for (uint32_t b = 0; b < 64; ++b)
            if (eval_state(n, b) != neg) tt |= 1ull << b;
        return tt;
    }

    // Splits a right operand (with a pending negation) into state conjuncts
    // and at most one nested temporal conjunct, pushing the negation inward.
    struct Conj {
        uint64_t P = ~0ull;
        int nested = -1;  // node of the nested F / G
        bool nested_neg = false;
    };
    bool split(int n, bool neg, Conj &c) const
    {
        const FNode &f = T[n];
        if (is_state(n)) { c.P &= table_of(n, neg); return true; }
        if ((f.kind == SMC_NODE_AND && !neg) || (f.kind == SMC_NODE_OR && neg))
            return split(f.c0, neg, c) && split(f.c1, neg, c);
        if (f.kind == SMC_NODE_IMPLIES && neg) return split(f.c0, false, c) && split(f.c1, true, c);
        if (f.kind == SMC_NODE_NOT) return split(f.c0, !neg, c);
        if (f.kind == SMC_NODE_EVENTUALLY || f.kind == SMC_NODE_ALWAYS) {
            if (c.nested >= 0) { err = "at most one nested F/G per operand"; return false; }
            c.nested = n;
            c.nested_neg = neg;
            return true;
        }
        err = "unsupported nesting of temporal operators in a right operand";
        return false;
    }

    // top-level leaf -> unit; returns the leaf's unit index, negated when the
    // unit is the F-form of a G.
    struct Leaf { int unit; bool neg; };
    std::vector<MonUnit> units;
    std::vector<Leaf> leaf_of;  // per node, or unit -1

    bool make_unit(int n, Leaf &leaf)
    {
        if ((int)units.size() >= SMC_MAX_UNITS) { err = "more than 4 temporal operators"; return false; }
        const FNode &f = T[n];
        MonUnit u;
        std::memset(&u, 0, sizeof(u));
        u.L = ~0ull;
        u.Q = ~0ull;
        bool neg_unit = false;
        Conj c;
        if (is_state(n)) {  // bare state formula: ff U[0,0] P
            u.L = 0;
            u.a = 0.0;
            u.b = 0.0;
            c.P = table_of(n, false);
        } else {
            if (!(f.lo >= 0.0) || !(f.hi >= f.lo) || std::isnan(f.hi) || std::isinf(f.lo)) {
                err = "interval must satisfy 0 <= lo <= hi";
                return false;
            }
            u.a = f.lo;
            u.b = f.hi;
            if (f.kind == SMC_NODE_NEXT) {  // X[a,b] psi: decided by the next state (nest 3)
                if (!is_state(f.c0)) { err = "the operand of X must be a state formula"; return false; }
                u.nest = 3;
                u.P = table_of(f.c0, false);
                leaf.unit = (int)units.size();
                leaf.neg = false;
                units.push_back(u);
                return true;
            }
            if (f.kind == SMC_NODE_UNTIL) {
                if (!is_state(f.c0)) { err = "left operand of U must be a state formula"; return false; }
                u.L = table_of(f.c0, false);
                if (!split(f.c1, false, c)) return false;
            } else if (f.kind == SMC_NODE_EVENTUALLY) {
                if (!split(f.c0, false, c)) return false;
            } else {  // G[a,b] psi = not F[a,b] not psi
                neg_unit = true;
                if (!split(f.c0, true, c)) return false;
            }
        }
        u.P = c.P;
        if (c.nested >= 0) {
            const FNode &g = T[c.nested];
            if (!is_state(g.c0)) { err = "nested F/G must have a state operand"; return false; }
            if (g.lo != 0.0 || !(g.hi >= 0.0) || std::isnan(g.hi)) {
                err = "nested F/G interval must be [0, d]";
                return false;
            }
            const bool eventually = (g.kind == SMC_NODE_EVENTUALLY) != c.nested_neg;
            u.nest = eventually ? 1 : 2;
            u.d = g.hi;
            u.Q = table_of(g.c0, c.nested_neg);
        }
        leaf.unit = (int)units.size();
        leaf.neg = neg_unit;
        units.push_back(u);
        return true;
    }

    // Kleene value of the top level given the unit values.
    int eval_top(int n, const int *val) const
    {
        const FNode &f = T[n];
        const Leaf &lf = leaf_of[n];
        if (lf.unit >= 0) return lf.neg ? kleene_not(val[lf.unit]) : val[lf.unit];
        switch (f.kind) {
        case SMC_NODE_NOT: return kleene_not(eval_top(f.c0, val));
        case SMC_NODE_AND: return kleene_and(eval_top(f.c0, val), eval_top(f.c1, val));
        case SMC_NODE_OR: return kleene_or(eval_top(f.c0, val), eval_top(f.c1, val));
        case SMC_NODE_IMPLIES:
            return kleene_or(kleene_not(eval_top(f.c0, val)), eval_top(f.c1, val));
        case SMC_NODE_TRUE: return V_T;
        case SMC_NODE_FALSE: return V_F;
        default: return V_U;
        }
    }

    bool top(int n)
    {
        const FNode &f = T[n];
        if (is_state(n) || is_temporal(f.kind)) {
            Leaf lf;
            if (!make_unit(n, lf)) return false;
            leaf_of[n] = lf;
            return true;
        }
        bool ok = true;
        if (f.c0 >= 0) ok = ok && top(f.c0);
        if (f.c1 >= 0) ok = ok && top(f.c1);
        return ok;
    }
};

void collect_atoms(const std::vector<FNode> &T, int n, std::vector<int> &bit, std::vector<int> &used)
{
    const FNode &f = T[n];
    if (f.kind == SMC_NODE_ATOM && bit[f.arg] < 0) {
        bit[f.arg] = (int)used.size();
        used.push_back(f.arg);
    }
    if (f.c0 >= 0) collect_atoms(T, f.c0, bit, used);
    if (f.c1 >= 0) collect_atoms(T, f.c1, bit, used);
}

}  // namespace

int parse_formula(const smc_node *nodes, int n_nodes, int n_atoms, std::vector<FNode> &tree,
                  int &root, std::string &err)
{
    tree.clear();
    std::vector<int> stack;
    if (!nodes || n_nodes <= 0) { err = "empty formula"; return SMC_E_INVALID_ARG; }
    for (int i = 0; i < n_nodes; ++i) {
        FNode f;
        f.kind = nodes[i].kind;
        f.arg = nodes[i].arg;
        f.lo = nodes[i].lo;
        f.hi = nodes[i].hi;
        int arity;
        switch (f.kind) {
        case SMC_NODE_TRUE: case SMC_NODE_FALSE: arity = 0; break;
        case SMC_NODE_ATOM:
            arity = 0;
            if (f.arg < 0 || f.arg >= n_atoms) { err = "atom index out of range"; return SMC_E_INVALID_ARG; }
            break;
        case SMC_NODE_NOT: case SMC_NODE_EVENTUALLY: case SMC_NODE_ALWAYS: case SMC_NODE_NEXT: arity = 1; break;
        case SMC_NODE_AND: case SMC_NODE_OR: case SMC_NODE_IMPLIES: case SMC_NODE_UNTIL: arity = 2; break;
        default: err = "unknown node kind"; return SMC_E_INVALID_ARG;
        }
        if ((int)stack.size() < arity) { err = "malformed postfix formula"; return SMC_E_INVALID_ARG; }
        if (arity == 2) {
            f.c1 = stack.back(); stack.pop_back();
            f.c0 = stack.back(); stack.pop_back();
        } else if (arity == 1) {
            f.c0 = stack.back(); stack.pop_back();
        }
        tree.push_back(f);
        stack.push_back((int)tree.size() - 1);
    }
    if (stack.size() != 1) { err = "malformed postfix formula"; return SMC_E_INVALID_ARG; }
    root = stack.back();
    return SMC_OK;
}

int compile_formula(const std::vector<FNode> &tree, int root, int n_atoms, double t_max,
                    MonProg &prog, std::vector<int> &used_atoms, std::string &err)
{
    std::memset(&prog, 0, sizeof(prog));
    std::vector<int> bit(n_atoms, -1);
    used_atoms.clear();
    collect_atoms(tree, root, bit, used_atoms);
    if ((int)used_atoms.size() > SMC_MAX_ATOMS) {
        err = "more than 6 distinct atoms";
        return SMC_E_UNSUPPORTED;
    }
    Compiler C(tree, err);
    C.atom_bit = bit;
    C.leaf_of.assign(tree.size(), Compiler::Leaf{-1, false});
    if (!C.top(root)) return SMC_E_UNSUPPORTED;
    const int nu = (int)C.units.size();
    prog.n_units = nu;
    prog.n_atoms = (int)used_atoms.size();
    for (int u = 0; u < nu; ++u) {
        prog.u[u] = C.units[u];
        const bool next = prog.u[u].nest == 3;  // decided by the first event, whatever its window
        if (!next && (std::isinf(prog.u[u].b) || (prog.u[u].nest && std::isinf(prog.u[u].d)))) prog.unbounded = 1;
        if (!next && prog.u[u].a > 0.0) prog.has_lower = 1;
    }
    if (prog.unbounded) {
        if (!(t_max > 0.0) || std::isinf(t_max)) {
            err = "unbounded formula needs a finite t_max_unbounded > 0";
            return SMC_E_INVALID_ARG;
        }
        prog.t_max = t_max;
    }
    int pw = 1;
    for (int u = 0; u < nu; ++u) pw *= 3;
    for (int idx = 0; idx < pw; ++idx) {
        int val[SMC_MAX_UNITS] = {0, 0, 0, 0};
        int r = idx;
        for (int u = 0; u < nu; ++u) { val[u] = r % 3; r /= 3; }
        prog.table[idx] = (uint8_t)C.eval_top(root, val);
    }
    return SMC_OK;
}

// The trace monitor's program (smc_nest.h): the formula tree renumbered
// from the root, atoms as bits of the used-atom vector, the static horizon
// (the latest time a position can matter: temporal operators add their
// interval end to their operands' horizons), the stopping time, and a memo
// column for each temporal node below another one (evaluated at many
// positions per check).
namespace {
// -1: too large (err says why), -2: a bad interval; under: a temporal
// operator is among the node's ancestors
int nest_copy(const std::vector<FNode> &T, int n, const std::vector<int> &bit, NestProg &np, int depth,
              bool under, std::string &err)
{
    if (depth > SMC_NEST_MAX_DEPTH) { err = "formula deeper than 10 nodes"; return -1; }
    if (np.n_nodes >= SMC_NEST_MAX_NODES) { err = "formula of more than 32 nodes"; return -1; }
    const FNode &f = T[n];
    const int id = np.n_nodes++;
    NestNode nd{};
    nd.kind = f.kind;
    nd.c0 = nd.c1 = -1;
    nd.bit = f.kind == SMC_NODE_ATOM ? bit[f.arg] : -1;
    nd.lo = f.lo;
    nd.hi = f.hi;
    const bool temporal = f.kind == SMC_NODE_UNTIL || f.kind == SMC_NODE_EVENTUALLY ||
                          f.kind == SMC_NODE_ALWAYS || f.kind == SMC_NODE_NEXT;
    if (temporal && !(f.lo >= 0.0 && std::isfinite(f.lo) && f.hi >= f.lo)) {
        err = "temporal interval needs 0 <= lo <= hi, lo finite";
        return -2;
    }
    nd.slot = (under && temporal && f.kind != SMC_NODE_NEXT) ? np.n_slots++ : -1;
    under = under || temporal;
    if (f.c0 >= 0 && (nd.c0 = nest_copy(T, f.c0, bit, np, depth + 1, under, err)) < 0) return nd.c0;
    if (f.c1 >= 0 && (nd.c1 = nest_copy(T, f.c1, bit, np, depth + 1, under, err)) < 0) return nd.c1;
    np.height = std::max(np.height, depth);
    np.nd[id] = nd;
    return id;
}

double nest_horizon(const NestProg &np, int n)
{
    const NestNode &f = np.nd[n];
    switch (f.kind) {
    case SMC_NODE_TRUE: case SMC_NODE_FALSE: case SMC_NODE_ATOM: return 0.0;
    case SMC_NODE_NOT: return nest_horizon(np, f.c0);
    case SMC_NODE_AND: case SMC_NODE_OR: case SMC_NODE_IMPLIES:
        return std::max(nest_horizon(np, f.c0), nest_horizon(np, f.c1));
    case SMC_NODE_UNTIL: return f.hi + std::max(nest_horizon(np, f.c0), nest_horizon(np, f.c1));
    default: return f.hi + nest_horizon(np, f.c0);
    }
}
}  // namespace

int compile_nested(const std::vector<FNode> &tree, int root, int n_atoms, double t_max, NestProg &np,
                   std::vector<int> &used_atoms, std::string &err)
{
    std::memset(&np, 0, sizeof(np));
    std::vector<int> bit(n_atoms, -1);
    used_atoms.clear();
    collect_atoms(tree, root, bit, used_atoms);
    if ((int)used_atoms.size() > SMC_MAX_ATOMS) {
        err = "more than 6 distinct atoms";
        return SMC_E_UNSUPPORTED;
    }
    const int rc = nest_copy(tree, root, bit, np, 1, false, err);
    if (rc == -2) return SMC_E_INVALID_ARG;
    if (rc < 0) return SMC_E_UNSUPPORTED;
    np.root = 0;
    np.t_static = nest_horizon(np, 0);
    if (std::isinf(np.t_static)) {
        if (!(t_max > 0.0) || std::isinf(t_max)) {
            err = "unbounded formula needs a finite t_max_unbounded > 0";
            return SMC_E_INVALID_ARG;
        }
        np.unbounded = 1;
        np.t_stop = t_max;
    } else {
        np.t_stop = np.t_static;
    }
    return SMC_OK;
}

// ---------------------------------------------------------------------------

namespace {
int64_t sat_floor(double b)
{
    const double lim = 4.0e18;
    if (b > lim) return (int64_t)lim;
    if (b < -lim) return -(int64_t)lim;
    return (int64_t)std::floor(b);
}
int64_t sat_ceil(double b)
{
    const double lim = 4.0e18;
    if (b > lim) return (int64_t)lim;
    if (b < -lim) return -(int64_t)lim;
    return (int64_t)std::ceil(b);
}
}  // namespace

void atom_threshold(int op, double b, int64_t &lo, int64_t &hi, bool &neg)
{
    const int64_t MIN = std::numeric_limits<int64_t>::min(), MAX = std::numeric_limits<int64_t>::max();
    neg = false;
    lo = MIN;
    hi = MAX;
    switch (op) {
    case SMC_OP_LT: hi = sat_ceil(b) - 1; break;   // L < b  <=>  L <= ceil(b) - 1
    case SMC_OP_LE: hi = sat_floor(b); break;      // L <= b <=>  L <= floor(b)
    case SMC_OP_GE: lo = sat_ceil(b); break;       // L >= b <=>  L >= ceil(b)
    case SMC_OP_GT: lo = sat_floor(b) + 1; break;  // L > b  <=>  L >= floor(b) + 1
    case SMC_OP_EQ:
    case SMC_OP_NE:
        if (std::floor(b) == b && std::fabs(b) <= 4.0e18) { lo = hi = (int64_t)b; }
        else { lo = 1; hi = 0; }  // never equal
        neg = (op == SMC_OP_NE);
        break;
    }
}

int validate_tokens(const smc_token *t, int n, int S, std::string &err)
{
    if (n < 1 || n > SMC_EXPR_MAX_TOKENS) { err = "an atom program needs 1..32 tokens"; return SMC_E_INVALID_ARG; }
    int d = 0;
    for (int i = 0; i < n; ++i) {
        switch (t[i].kind) {
        case SMC_TOK_SPECIES:
            if (t[i].arg < 0 || t[i].arg >= S) { err = "atom program: species out of range"; return SMC_E_INVALID_ARG; }
            ++d;
            break;
        case SMC_TOK_CONST:
            if (!std::isfinite(t[i].value)) { err = "atom program: constants must be finite"; return SMC_E_INVALID_ARG; }
            ++d;
            break;
        case SMC_TOK_ADD: case SMC_TOK_SUB: case SMC_TOK_MUL: case SMC_TOK_DIV:
            if (d < 2) { err = "atom program: operator without two operands"; return SMC_E_INVALID_ARG; }
            --d;
            break;
        case SMC_TOK_SQRT:
            if (d < 1) { err = "atom program: sqrt without an operand"; return SMC_E_INVALID_ARG; }
            break;
        case SMC_TOK_POWI:
            if (d < 1 || t[i].arg < 0 || t[i].arg > 16) { err = "atom program: bad power"; return SMC_E_INVALID_ARG; }
            break;
        default: err = "atom program: unknown token"; return SMC_E_INVALID_ARG;
        }
        if (d > SMC_EXPR_MAX_DEPTH) { err = "atom program deeper than 8"; return SMC_E_INVALID_ARG; }
    }
    if (d != 1) { err = "an atom program must leave one value"; return SMC_E_INVALID_ARG; }
    return SMC_OK;
}

double eval_tokens(const smc_token *t, int n, const int32_t *x)
{
    double st[SMC_EXPR_MAX_DEPTH + 1];
    int d = 0;
    for (int i = 0; i < n; ++i) {
        double b;
        switch (t[i].kind) {
        case SMC_TOK_SPECIES: st[d++] = (double)x[t[i].arg]; break;
        case SMC_TOK_CONST: st[d++] = t[i].value; break;
        case SMC_TOK_ADD: b = st[--d]; st[d - 1] = st[d - 1] + b; break;
        case SMC_TOK_SUB: b = st[--d]; st[d - 1] = st[d - 1] - b; break;
        case SMC_TOK_MUL: b = st[--d]; st[d - 1] = st[d - 1] * b; break;
        case SMC_TOK_DIV: b = st[--d]; st[d - 1] = st[d - 1] / b; break;
        case SMC_TOK_SQRT: st[d - 1] = std::sqrt(st[d - 1]); break;
        default: {
            const double a = st[d - 1];
            double r = 1.0;
            if (t[i].arg > 0) {
                r = a;
                for (int k = 1; k < t[i].arg; ++k) r = r * a;
            }
            st[d - 1] = r;
        }
        }
    }
    return st[0];
}

bool expr_atom_holds(const AtomExprView &e, const int32_t *x)
{
    const double l = eval_tokens(e.lhs, e.n_lhs, x), r = eval_tokens(e.rhs, e.n_rhs, x);
    switch (e.op) {
    case SMC_OP_LT: return l < r;
    case SMC_OP_LE: return l <= r;
    case SMC_OP_GE: return l >= r;
    case SMC_OP_GT: return l > r;
    case SMC_OP_EQ: return l == r;
    default: return l != r;
    }
}

int build_blob(const InstanceModel &M, int n_used, const int32_t *coef_used /*[n_used][S]*/,
               const int32_t *op_used, const double *bound_used, const AtomExprView *expr_used,
               std::vector<uint32_t> &blob, std::string &err)
{
    const int S = M.S, R = M.R;
    // stoichiometry CSR and changed-species sets
    std::vector<uint32_t> st_ptr(R + 1, 0), st;
    std::vector<std::vector<char>> changes(R, std::vector<char>(S, 0));
    for (int j = 0; j < R; ++j) {
        st_ptr[j] = (uint32_t)st.size();
        for (int i = 0; i < S; ++i) {
            const int32_t d = M.stoich[(size_t)j * S + i];
            if (d != 0) {
                st.push_back((uint32_t)i | ((uint32_t)d << 8));
                changes[j][i] = 1;
            }
        }
    }
    st_ptr[R] = (uint32_t)st.size();
    // propensity words: k | ra << 8 | rb << 16 | homo << 24, with species
    // index S standing for a constant-1 column, so h = x_ra (x_rb - homo) >> homo
    std::vector<uint32_t> pw(R);
    for (int k = 0; k < R; ++k) {
        int ra = M.reactants[2 * k], rb = M.reactants[2 * k + 1];
        if (ra < 0 && rb >= 0) { ra = rb; rb = -1; }
        uint32_t homo = 0;
        if (ra < 0) { ra = S; rb = S; }
        else if (rb < 0) rb = S;
        else if (ra == rb) homo = 1;
        pw[k] = (uint32_t)k | ((uint32_t)ra << 8) | ((uint32_t)rb << 16) | (homo << 24);
    }
    // rate-law factors: CSR by reaction (in the given order within a reaction)
    std::vector<uint32_t> f_ptr(R + 1, 0), f_words;
    std::vector<double> f_d;
    std::vector<float> f_f;
    std::vector<std::vector<int>> f_species(R);
    for (int k = 0; k < R; ++k) {
        f_ptr[k] = (uint32_t)f_words.size();
        for (int q = 0; q < M.n_fact; ++q) {
            if (M.f_reac[q] != k) continue;
            f_words.push_back((uint32_t)M.f_spec[q] | ((uint32_t)M.f_pow[q] << 8));
            for (int c = 0; c < 4; ++c) {
                f_d.push_back(M.f_par[4 * q + c]);
                f_f.push_back((float)M.f_par[4 * q + c]);
            }
            f_species[k].push_back(M.f_spec[q]);
            pw[k] |= SMC_PW_FACT;
        }
    }
    f_ptr[R] = (uint32_t)f_words.size();
    // dependency graph: k in dep(j) iff a_k reads a species that j changes
    std::vector<uint32_t> dep_ptr(R + 1, 0), dep;
    for (int j = 0; j < R; ++j) {
        dep_ptr[j] = (uint32_t)dep.size();
        for (int k = 0; k < R; ++k) {
            const int ra = M.reactants[2 * k], rb = M.reactants[2 * k + 1];
            bool reads = (ra >= 0 && changes[j][ra]) || (rb >= 0 && changes[j][rb]);
            for (int m : f_species[k]) reads = reads || changes[j][m];
            if (reads) dep.push_back(pw[k]);
        }
    }
    dep_ptr[R] = (uint32_t)dep.size();
    // atoms: sparse terms, thresholds, and which reactions move each atom
    std::vector<uint32_t> aterm_ptr(n_used + 1, 0), aterm, amask(R, 0);
    std::vector<int64_t> athr(2 * (size_t)n_used);
    uint32_t aneg = 0;
    for (int a = 0; a < n_used; ++a) {
        const int32_t *c = coef_used + (size_t)a * S;
        aterm_ptr[a] = (uint32_t)aterm.size();
        for (int i = 0; i < S; ++i) {
            if (c[i] > (1 << 20) || c[i] < -(1 << 20)) {
                err = "atom coefficients must lie in [-2^20, 2^20]";
                return SMC_E_INVALID_ARG;
            }
            if (c[i] != 0) aterm.push_back((uint32_t)i | ((uint32_t)c[i] << 8));
        }
        for (int j = 0; j < R; ++j) {
            int64_t d = 0;
            for (int i = 0; i < S; ++i) d += (int64_t)c[i] * M.stoich[(size_t)j * S + i];
            if (d != 0) amask[j] |= 1u << a;
        }
        if (expr_used && expr_used[a].op >= 0) {  // arithmetic atom: moved by any change of its species
            const AtomExprView &e = expr_used[a];
            for (int j = 0; j < R; ++j)
                for (int side = 0; side < 2; ++side) {
                    const smc_token *t = side ? e.rhs : e.lhs;
                    const int n = side ? e.n_rhs : e.n_lhs;
                    for (int i = 0; i < n; ++i)
                        if (t[i].kind == SMC_TOK_SPECIES && M.stoich[(size_t)j * S + t[i].arg] != 0)
                            amask[j] |= 1u << a;
                }
        }
        if (!std::isfinite(bound_used[a])) { err = "atom bounds must be finite"; return SMC_E_INVALID_ARG; }
        bool neg;
        atom_threshold(op_used[a], bound_used[a], athr[2 * a], athr[2 * a + 1], neg);
        if (neg) aneg |= 1u << a;
    }
    aterm_ptr[n_used] = (uint32_t)aterm.size();
    // layout
    blob.assign(BH_COUNT, 0);
    auto align2 = [&]() { if (blob.size() & 1) blob.push_back(0); };
    auto section = [&](int h) { align2(); blob[h] = (uint32_t)blob.size(); };
    section(BH_RATE_D);
    for (int k = 0; k < R; ++k) {
        uint32_t w[2];
        std::memcpy(w, &M.rates[k], 8);
        blob.push_back(w[0]);
        blob.push_back(w[1]);
    }
    section(BH_RATE_F);
    for (int k = 0; k < R; ++k) {
        const float f = (float)M.rates[k];
        uint32_t w;
        std::memcpy(&w, &f, 4);
        blob.push_back(w);
    }
    section(BH_REAC);
    blob.insert(blob.end(), pw.begin(), pw.end());
    section(BH_ST_PTR);
    blob.insert(blob.end(), st_ptr.begin(), st_ptr.end());
    section(BH_ST);
    blob.insert(blob.end(), st.begin(), st.end());
    section(BH_DEP_PTR);
    blob.insert(blob.end(), dep_ptr.begin(), dep_ptr.end());
    section(BH_DEP);
    blob.insert(blob.end(), dep.begin(), dep.end());
    section(BH_AMASK);
    blob.insert(blob.end(), amask.begin(), amask.end());
    section(BH_ATERM_PTR);
    blob.insert(blob.end(), aterm_ptr.begin(), aterm_ptr.end());
    section(BH_ATERM);
    blob.insert(blob.end(), aterm.begin(), aterm.end());
    bool small = S <= SMC_SMALL_MAX && R <= SMC_SMALL_MAX;
    for (size_t q = 0; q < st.size() && small; ++q) {
        const int32_t d = ((int32_t)st[q]) >> 8;
        if (d > 127 || d < -127) small = false;
    }
    if (small) {
        section(BH_DENSE);
        for (int j = 0; j < R; ++j) {
            uint32_t w[2] = {0, 0};
            for (int i = 0; i < S; ++i)
                w[i >> 2] |= ((uint32_t)(uint8_t)(int8_t)M.stoich[(size_t)j * S + i]) << (8 * (i & 3));
            blob.push_back(w[0]);
            blob.push_back(w[1]);
        }
    }
    section(BH_X0);
    for (int i = 0; i < S; ++i) blob.push_back((uint32_t)M.x0[i]);
    // arithmetic atoms' tokens (4 words each)
    std::vector<uint32_t> ex;
    std::vector<uint32_t> ex_off(n_used, 0);
    for (int a = 0; a < n_used; ++a) {
        if (!expr_used || expr_used[a].op < 0) continue;
        const AtomExprView &e = expr_used[a];
        ex_off[a] = (uint32_t)ex.size();
        for (int side = 0; side < 2; ++side) {
            const smc_token *t = side ? e.rhs : e.lhs;
            const int n = side ? e.n_rhs : e.n_lhs;
            for (int i = 0; i < n; ++i) {
                uint32_t w[2];
                std::memcpy(w, &t[i].value, 8);
                ex.push_back((uint32_t)t[i].kind | ((uint32_t)t[i].arg << 8));
                ex.push_back(0);
                ex.push_back(w[0]);
                ex.push_back(w[1]);
            }
        }
    }
    section(BH_ATOM);
    for (int a = 0; a < n_used; ++a) {
        if (expr_used && expr_used[a].op >= 0) {
            blob.push_back(SMC_ATOM_EXPR);
            blob.push_back((uint32_t)expr_used[a].op);
            blob.push_back(ex_off[a]);
            blob.push_back((uint32_t)expr_used[a].n_lhs);
            blob.push_back((uint32_t)expr_used[a].n_rhs);
            blob.push_back(0);
            continue;
        }
        const uint32_t nt = aterm_ptr[a + 1] - aterm_ptr[a];
        blob.push_back(nt == 1 ? aterm[aterm_ptr[a]] : 0xFFFFFFFFu);
        blob.push_back((aneg >> a) & 1u);
        for (int h = 0; h < 2; ++h) {
            const uint64_t v = (uint64_t)athr[2 * a + h];
            blob.push_back((uint32_t)v);
            blob.push_back((uint32_t)(v >> 32));
        }
    }
    if (!ex.empty()) {  // only read through arithmetic atoms' records
        section(BH_EXPR);
        blob.insert(blob.end(), ex.begin(), ex.end());
    }
    if (!f_words.empty()) {  // only read for reactions flagged SMC_PW_FACT
        section(BH_FACT_PTR);
        blob.insert(blob.end(), f_ptr.begin(), f_ptr.end());
        section(BH_FACT);
        blob.insert(blob.end(), f_words.begin(), f_words.end());
        section(BH_FACT_D);
        for (double v : f_d) {
            uint32_t w[2];
            std::memcpy(w, &v, 8);
            blob.push_back(w[0]);
            blob.push_back(w[1]);
        }
        section(BH_FACT_F);
        for (float v : f_f) {
            uint32_t w;
            std::memcpy(&w, &v, 4);
            blob.push_back(w);
        }
    }
    while (blob.size() & 3) blob.push_back(0);
    blob[BH_S] = (uint32_t)S;
    blob[BH_R] = (uint32_t)R;
    blob[BH_NA] = (uint32_t)n_used;
    blob[BH_WORDS] = (uint32_t)blob.size();
    return SMC_OK;
}

}  // namespace smc
