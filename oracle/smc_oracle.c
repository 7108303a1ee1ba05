/*
 * smc_oracle.c -- plain, slow, obviously correct CPU reference for the
 * statistical model checking hot path.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library links, loads or
 * calls this file; only the tests, the smoke check and the benchmark's CPU
 * baseline leg do.  It shares no code with the CUDA path.
 *
 * What it computes, each step following the paper (Ballarini et al.,
 * "Efficient Parallel Statistical Model Checking of Biochemical Networks"):
 *
 *  - Counter-based random numbers: Philox4x32-10 as defined by Salmon,
 *    Moraes, Dror and Shaw (SC'11), keyed by (seed) with the counter
 *    (event, trajectory, instance, 0).  The paper only asks for one seed per
 *    replica (Sec. 4); the counter keying replaces that seed stream.
 *  - The SSA direct method, Sec. 2.2 steps 1-5 with Eq. 1, 2a, 2b:
 *    propensities a_j = c_j * h_j(x) (times optional rational rate-law
 *    factors of single species, beyond the paper's mass action) recomputed
 *    from scratch every event,
 *    a_0 their left-to-right sum, tau = -ln(u_tau)/a_0, j the first index
 *    whose running sum exceeds u_j * a_0.
 *  - The full trace of the trajectory and the BLTLc semantics of Sec. 3.1
 *    evaluated on it by direct recursion (Kleene three-valued logic on a
 *    prefix, whose positions beyond the prefix are unknown), used both for
 *    the final verdict and for the on-the-fly stopping point of Sec. 3.2:
 *    a trajectory stops at the first prefix on which the formula is no
 *    longer undetermined.
 *  - The standard normal quantile by bisection on libm's erfc (used for the
 *    Wilson interval, Eq. 4, and sample size, Eq. 5, in oracle/wilson.py).
 *
 * Build: gcc -O2 -ffp-contract=off -fPIC -shared -pthread (no FMA
 * contraction, so every floating-point operation rounds once, in the
 * order written).
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------ */
/* Philox4x32-10 (Salmon et al. 2011): 10 rounds of two 32x32->64 multiplies
 * (multipliers 0xD2511F53 and 0xCD9E8D57), a word permutation with key
 * xor, and a Weyl key schedule (increments 0x9E3779B9, 0xBB67AE85).       */

void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)c0;
        uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        c0 = hi1 ^ c1 ^ k0;
        c1 = lo1;
        c2 = hi0 ^ c3 ^ k1;
        c3 = lo0;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* Uniform in the open interval (0,1): the top 52 bits of (hi:lo) plus one
 * half, times 2^-52.  (v + 0.5) needs at most 53 significant bits, so the
 * value is exact and lies in [2^-53, 1 - 2^-53]. */
double orc_u01(uint32_t hi, uint32_t lo)
{
    uint64_t v = ((((uint64_t)hi) << 32) | (uint64_t)lo) >> 12;
    return ((double)v + 0.5) * 0x1p-52;
}

/* ------------------------------------------------------------------------ */
/* model and formula                                                        */

typedef struct {
    int S, R;
    const int32_t *reactants; /* [R][2] species id or -1                    */
    const int32_t *stoich;    /* [R][S] net change                          */
    const double *rates;      /* [R]                                        */
    const int32_t *x0;        /* [S]                                        */
    /* rate-law factors (none for pure mass action): factor q multiplies the
     * propensity of reaction fr[q] by (a0 + a1 x^n) / (b0 + b1 x^n), x the
     * count of species fs[q], n = fn[q], (a0, a1, b0, b1) = fp[4q..4q+3]   */
    int n_fact;
    const int32_t *fr, *fs, *fn;
    const double *fp;
} orc_model;

enum { K_TRUE = 0, K_FALSE, K_ATOM, K_NOT, K_AND, K_OR, K_IMPLIES, K_UNTIL, K_EVENTUALLY, K_ALWAYS, K_NEXT };
enum { OP_LT = 0, OP_LE, OP_GE, OP_GT, OP_EQ, OP_NE };
enum { V_F = 0, V_T = 1, V_U = 2 }; /* Kleene truth values */

typedef struct {
    int32_t kind, c0, c1, arg; /* children (node indices) / atom index      */
    double lo, hi;             /* time interval [lo, hi] of U, F, G         */
} orc_node;

typedef struct {
    int32_t kind, arg; /* 0 species, 1 constant, 2 +, 3 -, 4 *, 5 /, 6 sqrt, 7 ^arg */
    double value;
} orc_token;

typedef struct {
    int n_nodes, root;
    const orc_node *nodes;
    int n_atoms, S;
    const int32_t *coef;  /* [n_atoms][S]                                   */
    const int32_t *op;    /* [n_atoms]                                      */
    const double *bound;  /* [n_atoms]                                      */
    /* arithmetic atoms (may be NULL): atom a is lhs <op> rhs when
     * expr_ptr[a + 1] > expr_ptr[a]; its tokens are tokens[expr_ptr[a] ..
     * expr_ptr[a + 1]), the first n_lhs[a] of them the left side           */
    const int32_t *expr_ptr, *n_lhs;
    const orc_token *tokens;
} orc_formula;

/* what is known about a path: positions 0..n-1 with entry times t[] and
 * states x[], and every later position (if any) has entry time >= tmin;
 * closed=1 means the path has no position beyond n-1 (absorbing state);
 * tmin_exact=1 means position n, if any, is entered exactly at tmin (its
 * entry time has been drawn).                                              */
typedef struct {
    int64_t n;
    const double *t;
    const int32_t *x;
    double tmin;
    int closed;
    int tmin_exact;
} orc_know;

static int not3(int a) { return a == V_U ? V_U : (a == V_T ? V_F : V_T); }
static int and3(int a, int b)
{
    if (a == V_F || b == V_F) return V_F;
    if (a == V_T && b == V_T) return V_T;
    return V_U;
}
static int or3(int a, int b)
{
    if (a == V_T || b == V_T) return V_T;
    if (a == V_F && b == V_F) return V_F;
    return V_U;
}

/* Sec. 3.1: sigma |= (val' <| val'') iff Eval(sigma[0], val') <| Eval(..). */
/* Sec. 3.1's Eval of an arithmetic value: a postfix program over the state,
 * every operation in double precision, rounded once; powers by repeated
 * multiplication. */
static double eval_value(const orc_token *tk, int n, const int32_t *x)
{
    double st[16];
    int d = 0;
    for (int i = 0; i < n; ++i) {
        const orc_token *t = tk + i;
        double b;
        switch (t->kind) {
        case 0: st[d++] = (double)x[t->arg]; break;
        case 1: st[d++] = t->value; break;
        case 2: b = st[--d]; st[d - 1] = st[d - 1] + b; break;
        case 3: b = st[--d]; st[d - 1] = st[d - 1] - b; break;
        case 4: b = st[--d]; st[d - 1] = st[d - 1] * b; break;
        case 5: b = st[--d]; st[d - 1] = st[d - 1] / b; break;
        case 6: st[d - 1] = sqrt(st[d - 1]); break;
        default: {
            const double a = st[d - 1];
            double r = 1.0;
            if (t->arg > 0) {
                r = a;
                for (int k = 1; k < t->arg; ++k) r = r * a;
            }
            st[d - 1] = r;
        }
        }
    }
    return st[0];
}

static int compare(int op, double v, double b)
{
    switch (op) {
    case OP_LT: return v < b;
    case OP_LE: return v <= b;
    case OP_GE: return v >= b;
    case OP_GT: return v > b;
    case OP_EQ: return v == b;
    default: return v != b;
    }
}

static int atom_holds(const orc_formula *f, int a, const int32_t *x)
{
    if (f->expr_ptr && f->expr_ptr[a + 1] > f->expr_ptr[a]) {
        const orc_token *tk = f->tokens + f->expr_ptr[a];
        const int nl = f->n_lhs[a], nr = f->expr_ptr[a + 1] - f->expr_ptr[a] - nl;
        return compare(f->op[a], eval_value(tk, nl, x), eval_value(tk + nl, nr, x));
    }
    int64_t L = 0;
    for (int i = 0; i < f->S; ++i) L += (int64_t)f->coef[(int64_t)a * f->S + i] * (int64_t)x[i];
    return compare(f->op[a], (double)L, f->bound[a]);
}

static int ev3(const orc_formula *f, int node, int64_t i, const orc_know *K);

/* sigma^i |= l U^[a,b] r  iff  exists j >= i with (t_j - t_i) in [a,b],
 * sigma^j |= r, and sigma^m |= l for all i <= m < j  (Sec. 3.1; the sum
 * of the sojourn times delta(sigma, m), i <= m < j, is the difference of
 * the entry times).  l = -1 stands for tt (F = tt U), neg_r evaluates
 * not r (used by G[a,b] r = not F[a,b] not r).                          */
static int until3(const orc_formula *f, int l, int r, int neg_r, double a, double b,
                  int64_t i, const orc_know *K)
{
    int acc = V_F, pre = V_T;
    for (int64_t j = i; j < K->n; ++j) {
        double dt = K->t[j] - K->t[i];
        if (dt > b) return acc; /* entry times never decrease along a path */
        if (dt >= a) {
            int rv = ev3(f, r, j, K);
            if (neg_r) rv = not3(rv);
            acc = or3(acc, and3(pre, rv));
            if (acc == V_T) return V_T;
        }
        int lv = (l < 0) ? V_T : ev3(f, l, j, K);
        pre = and3(pre, lv);
        if (pre == V_F) return acc;
    }
    /* unknown future positions: entry time >= tmin, any state */
    if (!K->closed && (K->tmin - K->t[i]) <= b) acc = or3(acc, and3(pre, V_U));
    return acc;
}

static int ev3(const orc_formula *f, int node, int64_t i, const orc_know *K)
{
    const orc_node *nd = &f->nodes[node];
    switch (nd->kind) {
    case K_TRUE: return V_T;
    case K_FALSE: return V_F;
    case K_ATOM: return atom_holds(f, nd->arg, K->x + i * f->S) ? V_T : V_F;
    case K_NOT: return not3(ev3(f, nd->c0, i, K));
    case K_AND: {
        int a = ev3(f, nd->c0, i, K);
        if (a == V_F) return V_F;
        return and3(a, ev3(f, nd->c1, i, K));
    }
    case K_OR: {
        int a = ev3(f, nd->c0, i, K);
        if (a == V_T) return V_T;
        return or3(a, ev3(f, nd->c1, i, K));
    }
    case K_IMPLIES: {
        int a = not3(ev3(f, nd->c0, i, K));
        if (a == V_T) return V_T;
        return or3(a, ev3(f, nd->c1, i, K));
    }
    case K_UNTIL: return until3(f, nd->c0, nd->c1, 0, nd->lo, nd->hi, i, K);
    case K_EVENTUALLY: return until3(f, -1, nd->c0, 0, nd->lo, nd->hi, i, K);
    case K_ALWAYS: return not3(until3(f, -1, nd->c0, 1, nd->lo, nd->hi, i, K));
    case K_NEXT: {  /* sigma^i |= X^I psi iff sigma^{i+1} |= psi and delta(sigma, i) in I */
        if (i + 1 < K->n) {
            const double d = K->t[i + 1] - K->t[i];
            if (d < nd->lo || d > nd->hi) return V_F;
            return ev3(f, nd->c0, i + 1, K);
        }
        if (K->closed) return V_F;
        const double d = K->tmin - K->t[i];
        if (d > nd->hi) return V_F;
        if (K->tmin_exact && d < nd->lo) return V_F;
        return V_U;
    }
    default: return V_U;
    }
}

/* Three-valued truth of the formula on a prefix (exported for tests). */
int orc_eval_prefix(const orc_formula *f, int64_t n, const double *t, const int32_t *x,
                    double tmin, int closed, int tmin_exact)
{
    orc_know K = {n, t, x, tmin, closed, tmin_exact};
    return ev3(f, f->root, 0, &K);
}

/* Latest time at which a position can still matter to the formula. */
static double static_horizon(const orc_formula *f, int node)
{
    const orc_node *nd = &f->nodes[node];
    switch (nd->kind) {
    case K_TRUE: case K_FALSE: case K_ATOM: return 0.0;
    case K_NOT: return static_horizon(f, nd->c0);
    case K_AND: case K_OR: case K_IMPLIES: {
        double a = static_horizon(f, nd->c0), b = static_horizon(f, nd->c1);
        return a > b ? a : b;
    }
    case K_UNTIL: {
        double a = static_horizon(f, nd->c0), b = static_horizon(f, nd->c1);
        return nd->hi + (a > b ? a : b);
    }
    default: return nd->hi + static_horizon(f, nd->c0);
    }
}

/* ------------------------------------------------------------------------ */
/* one trajectory                                                            */

typedef struct {
    double *t;
    int32_t *x;
    int64_t cap;
    double *a; /* propensities, [R] */
} orc_buf;

static int buf_reserve(orc_buf *B, int64_t n, int S)
{
    if (n <= B->cap) return 0;
    int64_t c = B->cap ? B->cap : 1024;
    while (c < n) c *= 2;
    double *t = (double *)realloc(B->t, (size_t)c * sizeof(double));
    if (!t) return -1;
    B->t = t;
    int32_t *x = (int32_t *)realloc(B->x, (size_t)c * (size_t)S * sizeof(int32_t));
    if (!x) return -1;
    B->x = x;
    B->cap = c;
    return 0;
}

typedef struct {
    uint8_t verdict; /* 1 = the path satisfies the formula                  */
    uint8_t status;  /* 0 = decided, 1 = event budget exhausted, 2 = error  */
    uint64_t events; /* reactions fired before the verdict was fixed        */
    double t_final;  /* entry time of the last state entered                */
} orc_result;

/* Sec. 2.2: a_j(x) = c_j * h_j(x), h_j the number of distinct reactant
 * combinations: 1 (no reactant), x_a, x_a * x_b, or x_a (x_a - 1) / 2 for
 * a homodimer S_a + S_a.  h_j is an exact integer, rounded once to double. */
static double propensity(const orc_model *M, int j, const int32_t *x)
{
    int ra = M->reactants[2 * j], rb = M->reactants[2 * j + 1];
    int64_t h;
    if (ra < 0 && rb < 0) h = 1;
    else if (rb < 0) h = x[ra];
    else if (ra < 0) h = x[rb];
    else if (ra == rb) h = (int64_t)x[ra] * ((int64_t)x[ra] - 1) / 2;
    else h = (int64_t)x[ra] * (int64_t)x[rb];
    double a = M->rates[j] * (double)h;
    /* rate-law factors of reaction j, in the order given: x^n by repeated
     * multiplication, then numerator, denominator, their quotient, and the
     * product with the propensity, each rounded once */
    for (int q = 0; q < M->n_fact; ++q) {
        if (M->fr[q] != j) continue;
        const double xv = (double)x[M->fs[q]];
        double xn = xv;
        for (int i = 1; i < M->fn[q]; ++i) xn = xn * xv;
        const double *c = M->fp + 4 * q;
        const double num = c[0] + c[1] * xn;
        const double den = c[2] + c[3] * xn;
        a = a * (num / den);
    }
    return a;
}

/* knowledge point q: q = 2k -> positions 0..k known, tmin = t_k;
 * q = 2k+1 -> positions 0..k known, tmin = entry time of position k+1
 * (drawn, not yet applied) or closed when the path absorbed after k.      */
typedef struct {
    const orc_formula *f;
    const double *t;
    const int32_t *x;
    int64_t E;        /* last simulated position                            */
    double tnext;     /* entry time drawn after position E (if drawn)       */
    int have_next;    /* 1: tnext valid, 2: absorbed after E, 0: neither    */
} orc_path;

static int eval_at(const orc_path *P, int64_t q)
{
    int64_t k = q / 2;
    orc_know K;
    K.n = k + 1;
    K.t = P->t;
    K.x = P->x;
    K.closed = 0;
    K.tmin_exact = (int)(q & 1);  /* after a draw the next entry time is known */
    if ((q & 1) == 0) {
        K.tmin = P->t[k];
    } else if (k < P->E) {
        K.tmin = P->t[k + 1];
    } else if (P->have_next == 2) {
        K.tmin = INFINITY;
        K.closed = 1;
    } else {
        K.tmin = P->tnext;
    }
    return ev3(P->f, P->f->root, 0, &K);
}

static void run_one(const orc_model *M, const orc_formula *f, uint64_t seed, uint32_t instance,
                    uint64_t traj, uint64_t budget, double t_max, orc_buf *B, orc_result *res,
                    int32_t *x_final)
{
    const int S = M->S, R = M->R;
    const uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    double T_static = static_horizon(f, f->root);
    double T_stop = isfinite(T_static) ? T_static : t_max;

    if (buf_reserve(B, 1, S)) { res->status = 2; return; }
    memcpy(B->x, M->x0, (size_t)S * sizeof(int32_t));
    B->t[0] = 0.0;

    orc_path P = {f, NULL, NULL, 0, 0.0, 0};
    int64_t E = 0;
    int64_t q_lo = -1, q_hi = -1; /* last undecided / first decided known   */
    int64_t next_check = 0;
    int pessimistic = 0;

    for (;;) {
        P.t = B->t; P.x = B->x; P.E = E; P.have_next = 0;
        if (E == next_check) { /* doubling schedule of checks at q = 2E    */
            if (eval_at(&P, 2 * E) != V_U) { q_hi = 2 * E; break; }
            q_lo = 2 * E;
            next_check = next_check ? 2 * next_check : 1;
        }
        if ((uint64_t)E >= budget) { /* no further event may fire */
            if (q_lo < 2 * E && eval_at(&P, 2 * E) != V_U) q_hi = 2 * E;
            break;
        }

        /* Step 1: a_0 = sum_j a_j, left to right. */
        const int32_t *x = B->x + E * S;
        double a0 = 0.0;
        for (int j = 0; j < R; ++j) { B->a[j] = propensity(M, j, x); a0 += B->a[j]; }
        if (!(a0 > 0.0)) { /* absorbing state: no position after E */
            P.have_next = 2;
            q_hi = 2 * E + 1;
            break;
        }
        /* Eq. 2a, 2b from one Philox block keyed by (event, trajectory, instance). */
        uint32_t ctr[4] = {(uint32_t)E, (uint32_t)traj, instance, 0u}, w[4];
        orc_philox4x32_10(ctr, key, w);
        double u_tau = orc_u01(w[0], w[1]);
        double u_sel = orc_u01(w[2], w[3]);
        double tau = -log(u_tau) / a0;
        double tnext = B->t[E] + tau;
        if (tnext > T_stop) {
            P.tnext = tnext; P.have_next = 1;
            int v = eval_at(&P, 2 * E + 1);
            if (v != V_U) { q_hi = 2 * E + 1; break; }
            if (!isfinite(T_static)) { pessimistic = 1; q_hi = 2 * E + 1; break; }
            if (tnext > 4.0 * T_stop + 1.0) { res->status = 2; return; }
        }
        double r = u_sel * a0, cum = 0.0;
        int jsel = -1, jlast = -1;
        for (int j = 0; j < R; ++j) {
            cum += B->a[j];
            if (B->a[j] > 0.0) jlast = j;
            if (cum > r) { jsel = j; break; }
        }
        if (jsel < 0) jsel = jlast; /* rounding: r reached the full sum */
        if (buf_reserve(B, E + 2, S)) { res->status = 2; return; }
        const int32_t *xs = B->x + E * S;
        int32_t *xn = B->x + (E + 1) * S;
        for (int i = 0; i < S; ++i) xn[i] = xs[i] + M->stoich[(int64_t)jsel * S + i];
        B->t[E + 1] = tnext;
        ++E;
    }
    P.t = B->t; P.x = B->x; P.E = E;
    if (q_hi < 0) { /* budget exhausted without a verdict */
        res->status = 1;
        res->verdict = 0;
        res->events = (uint64_t)E;
        res->t_final = B->t[E];
        if (x_final) memcpy(x_final, B->x + E * S, (size_t)S * sizeof(int32_t));
        return;
    }
    /* first decided knowledge point in (q_lo, q_hi]: decidedness is monotone */
    int64_t lo = q_lo, hi = q_hi;
    while (hi - lo > 1) {
        int64_t mid = lo + (hi - lo) / 2;
        if (eval_at(&P, mid) != V_U) hi = mid; else lo = mid;
    }
    int v = eval_at(&P, hi);
    if (v == V_U) v = pessimistic ? V_F : V_U;
    int64_t k = hi / 2;
    res->status = (v == V_U) ? 2 : 0;
    res->verdict = (v == V_T);
    res->events = (uint64_t)k;
    res->t_final = B->t[k];
    if (x_final) memcpy(x_final, B->x + k * S, (size_t)S * sizeof(int32_t));
}

/* ------------------------------------------------------------------------ */
/* trajectory ranges over threads                                            */

typedef struct {
    const orc_model *M;
    const orc_formula *f;
    uint64_t seed, traj_begin, n_traj, budget;
    uint32_t instance;
    double t_max;
    uint8_t *verdict, *status;
    uint64_t *events;
    double *t_final;
    int32_t *x_final;
    int64_t next;
    pthread_mutex_t mu;
    int failed;
} orc_job;

static void *worker(void *arg)
{
    orc_job *J = (orc_job *)arg;
    orc_buf B = {NULL, NULL, 0, NULL};
    B.a = (double *)malloc((size_t)(J->M->R > 0 ? J->M->R : 1) * sizeof(double));
    if (!B.a) { J->failed = 1; return NULL; }
    for (;;) {
        pthread_mutex_lock(&J->mu);
        int64_t i0 = J->next;
        J->next += 8;
        pthread_mutex_unlock(&J->mu);
        if ((uint64_t)i0 >= J->n_traj) break;
        int64_t i1 = i0 + 8;
        if ((uint64_t)i1 > J->n_traj) i1 = (int64_t)J->n_traj;
        for (int64_t i = i0; i < i1; ++i) {
            orc_result r = {0, 0, 0, 0.0};
            run_one(J->M, J->f, J->seed, J->instance, J->traj_begin + (uint64_t)i, J->budget,
                    J->t_max, &B, &r, J->x_final ? J->x_final + i * J->M->S : NULL);
            if (J->verdict) J->verdict[i] = r.verdict;
            if (J->status) J->status[i] = r.status;
            if (J->events) J->events[i] = r.events;
            if (J->t_final) J->t_final[i] = r.t_final;
            if (r.status == 2) J->failed = 1;
        }
    }
    free(B.t); free(B.x); free(B.a);
    return NULL;
}

/* Runs trajectories traj_begin .. traj_begin+n_traj-1 of one instance.
 * Output arrays (any may be NULL) have n_traj entries (x_final: n_traj*S).
 * Returns 0, or -1 if a trajectory failed (allocation, undecided path).  */
int orc_run(int S, int R, const int32_t *reactants, const int32_t *stoich, const double *rates,
            const int32_t *x0, int n_fact, const int32_t *fact_reaction, const int32_t *fact_species,
            const int32_t *fact_power, const double *fact_param, int n_nodes, int root,
            const orc_node *nodes, int n_atoms, const int32_t *coef, const int32_t *op,
            const double *bound, const int32_t *expr_ptr, const int32_t *expr_n_lhs,
            const orc_token *expr_tokens, uint64_t seed, uint32_t instance, uint64_t traj_begin, uint64_t n_traj,
            uint64_t budget, double t_max, int n_threads, uint8_t *verdict, uint8_t *status,
            uint64_t *events, double *t_final, int32_t *x_final)
{
    orc_model M = {S, R, reactants, stoich, rates, x0, n_fact, fact_reaction, fact_species, fact_power,
                   fact_param};
    orc_formula f = {n_nodes, root, nodes, n_atoms, S, coef, op, bound, expr_ptr, expr_n_lhs, expr_tokens};
    orc_job J;
    memset(&J, 0, sizeof(J));
    J.M = &M; J.f = &f; J.seed = seed; J.traj_begin = traj_begin; J.n_traj = n_traj;
    J.budget = budget; J.instance = instance; J.t_max = t_max;
    J.verdict = verdict; J.status = status; J.events = events; J.t_final = t_final;
    J.x_final = x_final;
    pthread_mutex_init(&J.mu, NULL);
    if (n_threads < 1) n_threads = 1;
    if (n_threads > 256) n_threads = 256;
    pthread_t th[256];
    int started = 0;
    for (int i = 1; i < n_threads; ++i)
        if (pthread_create(&th[started], NULL, worker, &J) == 0) ++started;
    worker(&J);
    for (int i = 0; i < started; ++i) pthread_join(th[i], NULL);
    pthread_mutex_destroy(&J.mu);
    return J.failed ? -1 : 0;
}

/* ------------------------------------------------------------------------ */
/* standard normal quantile: the z with Phi(z) = p.  For p > 1/2 the upper
 * tail Q(z) = erfc(z/sqrt2)/2 = 1 - p is solved instead (1 - p is exact
 * there, and erfc keeps full relative precision in the tail); bisection to
 * the last representable double.                                           */
double orc_normal_quantile(double p)
{
    if (!(p > 0.0 && p < 1.0)) return NAN;
    int upper = p > 0.5;
    double target = upper ? 1.0 - p : p;   /* tail probability, <= 1/2      */
    double sgn = upper ? 1.0 : -1.0;       /* z = sgn * w with w >= 0        */
    double lo = 0.0, hi = 40.0;            /* tail(w) = erfc(w/sqrt2)/2 falls */
    for (int it = 0; it < 4000; ++it) {
        double mid = 0.5 * (lo + hi);
        if (mid == lo || mid == hi) break;
        double tail = 0.5 * erfc(mid / sqrt(2.0));
        if (tail > target) lo = mid; else hi = mid;
    }
    double tl = 0.5 * erfc(lo / sqrt(2.0)), th = 0.5 * erfc(hi / sqrt(2.0));
    double w = (fabs(tl - target) <= fabs(th - target)) ? lo : hi;
    return sgn * w;
}
