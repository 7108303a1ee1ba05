// Host driver for the kernels' linear atoms: builds an instance table with
// the library's build_blob (smc_compile.cpp) and evaluates atom_bit of
// paper_0912_2551_gb300/csrc/smc_device.cuh (compiled for the host through
// host_cuda_shims.h) on given states.  Input: S n_atoms; per atom op bound
// coef[S]; then states x[S] until end of input.  Output per state: the
// atom bit vector, for tests/test_atom_device_host.py.
#include <stdio.h>

#include <string>
#include <vector>

#include "host_cuda_shims.h"
#include "smc.h"
#include "smc_compile.h"
#include "smc_device.cuh"

int main()
{
    int S, NA;
    if (scanf("%d %d", &S, &NA) != 2) return 2;
    std::vector<int32_t> coef((size_t)NA * S), op(NA);
    std::vector<double> bound(NA);
    for (int a = 0; a < NA; ++a) {
        if (scanf("%d %lf", &op[a], &bound[a]) != 2) return 2;
        for (int i = 0; i < S; ++i) if (scanf("%d", &coef[(size_t)a * S + i]) != 1) return 2;
    }
    // a one-reaction network (0 -> species 0): only the atom sections matter
    std::vector<int32_t> reac = {-1, -1}, st(S, 0), x0(S, 0);
    st[0] = 1;
    const double rate = 1.0;
    smc::InstanceModel M;
    M.S = S;
    M.R = 1;
    M.reactants = reac.data();
    M.stoich = st.data();
    M.rates = &rate;
    M.x0 = x0.data();
    std::vector<uint32_t> blob;
    std::string err;
    if (smc::build_blob(M, NA, coef.data(), op.data(), bound.data(), nullptr, blob, err) != SMC_OK) {
        printf("error %s\n", err.c_str());
        return 1;
    }
    const uint32_t *atoms = blob.data() + blob[BH_ATOM], *tptr = blob.data() + blob[BH_ATERM_PTR];
    const uint32_t *terms = blob.data() + blob[BH_ATERM];
    std::vector<int32_t> xs((size_t)S * 32, 0);  // lane-minor state, lane 0
    for (;;) {
        for (int i = 0; i < S; ++i)
            if (scanf("%d", &xs[(size_t)i * 32]) != 1) return 0;
        uint32_t bits = 0;
        for (int a = 0; a < NA; ++a) bits |= atom_bit<false>(atoms, tptr, terms, nullptr, xs.data(), a);
        printf("%u\n", bits);
    }
}
