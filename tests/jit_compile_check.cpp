// Host check that the model-specialized kernels compile: for a few network
// structures (small, with rate-law factors, with an arithmetic atom, medium)
// the library writes the model header and NVRTC compiles the kernels for
// sm_103a.  Without a GPU the library then fails to load the cubin; that
// failure, not a compile error, is what this check expects there.  Prints
// one line per case, "case=<name> compiled=<0|1>", and exits 0 when all
// compiled.
#include <stdio.h>

#include <string>
#include <vector>

#include "smc.h"
#include "smc_jit.h"

using namespace smc;

static bool compiled(const JitModel &M, const char *name)
{
    std::string why;
    const std::string h = jit_model_header(M, why);
    if (h.empty()) {
        printf("case=%s compiled=0 reason=%s\n", name, why.c_str());
        return false;
    }
    JitKernels k;
    std::string err;
    const int rc = jit_compile(h, k, err);
    const bool ok = rc == 0 || err.rfind("cudaLibrary", 0) == 0;  // compiled; loading needs a GPU
    printf("case=%s compiled=%d%s%s\n", name, (int)ok, ok ? "" : " error=", ok ? "" : err.substr(0, 400).c_str());
    return ok;
}

int main()
{
    bool all = true;
    // Lotka-Volterra: X -> 2X, X + Y -> 2Y, Y -> 0; atoms X > 0, Y > 0
    const int32_t reac[] = {0, -1, 0, 1, 1, -1};
    const int32_t st[] = {1, 0, -1, 1, 0, -1};
    const int32_t coef[] = {1, 0, 0, 1};
    const int64_t lo[] = {1, 1}, hi[] = {(int64_t)1 << 40, (int64_t)1 << 40};
    const uint8_t neg[] = {0, 0};
    JitModel lv;
    lv.S = 2;
    lv.R = 3;
    lv.reactants = reac;
    lv.stoich = st;
    lv.n_atoms = 2;
    lv.coef = coef;
    lv.lo = lo;
    lv.hi = hi;
    lv.neg = neg;
    all &= compiled(lv, "lotka_volterra");
    // a Hill factor (x_1^2 / (K + x_1^2)) on the first reaction
    const int32_t fr[] = {0}, fs[] = {1}, fp[] = {2};
    const double fpar[] = {0.0, 1.0, 400.0, 1.0};
    JitModel fa = lv;
    fa.n_fact = 1;
    fa.f_reac = fr;
    fa.f_spec = fs;
    fa.f_pow = fp;
    fa.f_par = fpar;
    all &= compiled(fa, "rate_law_factor");
    // atom 1 as sqrt(x0 x1) <= 700 (an arithmetic atom)
    const smc_token lhs[] = {{SMC_TOK_SPECIES, 0, 0.0}, {SMC_TOK_SPECIES, 1, 0.0}, {SMC_TOK_MUL, 0, 0.0},
                             {SMC_TOK_SQRT, 0, 0.0}};
    const smc_token rhs[] = {{SMC_TOK_CONST, 0, 700.0}};
    AtomExprView ex[2];
    ex[1].op = SMC_OP_LE;
    ex[1].lhs = lhs;
    ex[1].n_lhs = 4;
    ex[1].rhs = rhs;
    ex[1].n_rhs = 1;
    JitModel ea = lv;
    ea.expr = ex;
    all &= compiled(ea, "arithmetic_atom");
    // a medium network: 22 species, 30 reactions (enzymatic steps), one atom
    const int S = 22, R = 30;
    std::vector<int32_t> mr(2 * R, -1), ms(R * S, 0), mc(S, 0);
    for (int k = 0; k < R; ++k) {
        mr[2 * k] = k % S;
        if (k % 3 == 0) mr[2 * k + 1] = (k + 5) % S;
        ms[k * S + k % S] = -1;
        ms[k * S + (k + 7) % S] = 1;
    }
    mc[10] = 1;
    const int64_t mlo[] = {500}, mhi[] = {(int64_t)1 << 40};
    const uint8_t mneg[] = {0};
    JitModel md;
    md.S = S;
    md.R = R;
    md.reactants = mr.data();
    md.stoich = ms.data();
    md.n_atoms = 1;
    md.coef = mc.data();
    md.lo = mlo;
    md.hi = mhi;
    md.neg = mneg;
    all &= compiled(md, "medium_22x30");
    return all ? 0 : 1;
}
