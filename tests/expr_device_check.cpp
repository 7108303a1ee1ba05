// Host driver for the kernels' arithmetic atoms (eval_expr and
// expr_atom_bit of paper_0912_2551_gb300/csrc/smc_device.cuh, compiled for
// the host through host_cuda_shims.h), with the tokens in the instance
// table's encoding (kind | arg << 8, 0, the constant's two words).  Input:
// S, then cases until end of input: op n_lhs n_rhs, the tokens (kind arg
// value), the state x[S].  Output per case: the two sides' bit patterns
// (hex) and the atom's bit, for tests/test_expr_device_host.py.
#include <inttypes.h>
#include <stdio.h>

#include <vector>

#include "host_cuda_shims.h"
#include "smc_device.cuh"

int main()
{
    int S;
    if (scanf("%d", &S) != 1) return 2;
    for (;;) {
        int op, nl, nr;
        if (scanf("%d %d %d", &op, &nl, &nr) != 3) return 0;
        std::vector<uint32_t> ex(4 * (size_t)(nl + nr));
        for (int i = 0; i < nl + nr; ++i) {
            int kind, arg;
            double v;
            if (scanf("%d %d %lf", &kind, &arg, &v) != 3) return 2;
            uint32_t w[2];
            memcpy(w, &v, 8);
            ex[4 * i] = (uint32_t)kind | ((uint32_t)arg << 8);
            ex[4 * i + 1] = 0;
            ex[4 * i + 2] = w[0];
            ex[4 * i + 3] = w[1];
        }
        std::vector<int32_t> xs((size_t)S * 32, 0);  // lane-minor state, lane 0
        for (int i = 0; i < S; ++i)
            if (scanf("%d", &xs[(size_t)i * 32]) != 1) return 2;
        const uint32_t A[6] = {SMC_ATOM_EXPR, (uint32_t)op, 0u, (uint32_t)nl, (uint32_t)nr, 0u};
        const double l = eval_expr(ex.data(), nl, xs.data()), r = eval_expr(ex.data() + 4 * nl, nr, xs.data());
        uint64_t bl, br;
        memcpy(&bl, &l, 8);
        memcpy(&br, &r, 8);
        printf("%016" PRIx64 " %016" PRIx64 " %u\n", bl, br, expr_atom_bit(A, ex.data(), xs.data()));
    }
}
