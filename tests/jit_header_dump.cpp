// Host driver: writes the model header that the library generates for its
// model-specialized kernels (jit_model_header in
// paper_0912_2551_gb300/csrc/smc_jit.cpp) for one network read from
// standard input, for tests/test_jit_host_eval.py.
// Input: S R n_atoms n_factors; reactants [R][2]; stoich [R][S]; per atom
// coef[S] lo hi neg; per factor reaction species power a0 a1 b0 b1.
#include <stdint.h>
#include <stdio.h>

#include <string>
#include <vector>

#include "smc.h"
#include "smc_jit.h"

int main()
{
    int S, R, NA, NF;
    if (scanf("%d %d %d %d", &S, &R, &NA, &NF) != 4) return 2;
    std::vector<int32_t> reac(2 * R), st((size_t)R * S), coef((size_t)NA * S), fr(NF), fs(NF), fp(NF);
    std::vector<int64_t> lo(NA), hi(NA);
    std::vector<uint8_t> neg(NA);
    std::vector<double> par(4 * (size_t)NF);
    for (auto &v : reac) if (scanf("%d", &v) != 1) return 2;
    for (auto &v : st) if (scanf("%d", &v) != 1) return 2;
    for (int a = 0; a < NA; ++a) {
        for (int i = 0; i < S; ++i) if (scanf("%d", &coef[(size_t)a * S + i]) != 1) return 2;
        long long l, h;
        int n;
        if (scanf("%lld %lld %d", &l, &h, &n) != 3) return 2;
        lo[a] = l;
        hi[a] = h;
        neg[a] = (uint8_t)n;
    }
    for (int q = 0; q < NF; ++q) {
        if (scanf("%d %d %d", &fr[q], &fs[q], &fp[q]) != 3) return 2;
        for (int c = 0; c < 4; ++c) if (scanf("%lf", &par[4 * q + c]) != 1) return 2;
    }
    smc::JitModel M;
    M.S = S;
    M.R = R;
    M.reactants = reac.data();
    M.stoich = st.data();
    M.n_atoms = NA;
    M.coef = coef.data();
    M.lo = lo.data();
    M.hi = hi.data();
    M.neg = neg.data();
    M.n_fact = NF;
    M.f_reac = fr.data();
    M.f_spec = fs.data();
    M.f_pow = fp.data();
    M.f_par = par.data();
    std::string why;
    const std::string h = smc::jit_model_header(M, why);
    if (h.empty()) {
        fprintf(stderr, "not eligible: %s\n", why.c_str());
        return 1;
    }
    fputs(h.c_str(), stdout);
    return 0;
}
