// Host driver for the instance-table builder build_blob of
// paper_0912_2551_gb300/csrc/smc_compile.cpp: reads one network, its atoms
// and rate-law factors from standard input and prints the table's 32-bit
// words (decimal, one line) for tests/test_blob_host.py to decode.
// Input (whitespace separated): S R n_atoms n_factors; reactants [R][2];
// stoich [R][S]; rates [R]; x0 [S]; per atom: op bound coef[S]; per factor:
// reaction species power a0 a1 b0 b1.
#include <stdint.h>
#include <stdio.h>

#include <string>
#include <vector>

#include "smc.h"
#include "smc_compile.h"

int main()
{
    int S, R, NA, NF;
    if (scanf("%d %d %d %d", &S, &R, &NA, &NF) != 4) return 2;
    std::vector<int32_t> reac(2 * R), st((size_t)R * S), x0(S), coef((size_t)NA * S), op(NA), f_reac(NF),
        f_spec(NF), f_pow(NF);
    std::vector<double> rates(R), bound(NA), f_par(4 * (size_t)NF);
    for (auto &v : reac) if (scanf("%d", &v) != 1) return 2;
    for (auto &v : st) if (scanf("%d", &v) != 1) return 2;
    for (auto &v : rates) if (scanf("%lf", &v) != 1) return 2;
    for (auto &v : x0) if (scanf("%d", &v) != 1) return 2;
    for (int a = 0; a < NA; ++a) {
        if (scanf("%d %lf", &op[a], &bound[a]) != 2) return 2;
        for (int i = 0; i < S; ++i) if (scanf("%d", &coef[(size_t)a * S + i]) != 1) return 2;
    }
    for (int q = 0; q < NF; ++q) {
        if (scanf("%d %d %d", &f_reac[q], &f_spec[q], &f_pow[q]) != 3) return 2;
        for (int c = 0; c < 4; ++c) if (scanf("%lf", &f_par[4 * q + c]) != 1) return 2;
    }
    smc::InstanceModel M;
    M.S = S;
    M.R = R;
    M.reactants = reac.data();
    M.stoich = st.data();
    M.rates = rates.data();
    M.x0 = x0.data();
    M.n_fact = NF;
    M.f_reac = f_reac.data();
    M.f_spec = f_spec.data();
    M.f_pow = f_pow.data();
    M.f_par = f_par.data();
    std::vector<uint32_t> blob;
    std::string err;
    const int rc = smc::build_blob(M, NA, coef.data(), op.data(), bound.data(), nullptr, blob, err);
    if (rc != SMC_OK) {
        printf("error %d %s\n", rc, err.c_str());
        return 1;
    }
    for (size_t i = 0; i < blob.size(); ++i) printf(i ? " %u" : "%u", blob[i]);
    printf("\n");
    return 0;
}
