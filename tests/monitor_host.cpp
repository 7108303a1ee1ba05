// Host replay of the compiled BLTLc monitor: the device code of
// paper_0912_2551_gb300/csrc/smc_device.cuh (mon_start, mon_state,
// mon_draw, mon_close), compiled for the host with the CUDA intrinsics it
// names replaced by the operations they denote, driven over given paths in
// the order the SSA kernels use (as the library's replay kernel does), with
// the monitor program and atom thresholds from the library's compiler
// (smc_compile.cpp).  tests/test_monitor_host.py compares the verdicts and
// the points where they become fixed with the oracle's trace semantics.
// Input: S n_atoms n_nodes; per atom op bound coef[S]; per node kind arg lo
// hi; n_paths; per path len closed tmin, then len x [S] and len t.
// Output: one line "verdict decided_at" per path (verdict 0 undetermined,
// 1 false, 2 true).  As the library does, a formula outside the monitor's
// fragment goes to the trace monitor (smc_nest.h: the path's states and
// entry times recorded, the verdict and its decision point computed from
// them); with the argument "nest" every formula does, and with "memo" every
// formula goes to the trace monitor with its memo, run as the SSA kernel
// runs it: positions recorded in order (their memo cells zeroed), the
// formula evaluated at every knowledge point in turn, each result checked
// against the evaluation without the memo (exit status 3 on a mismatch);
// "memo_sparse" the same at a pseudo-random third of the knowledge points
// (the last one always), as the kernel's checks skip most of them.
#include <math.h>
#include <stdint.h>
#include <stdio.h>
#include <string.h>

#include <string>
#include <vector>

#include "host_cuda_shims.h"
#include "smc.h"
#include "smc_compile.h"
#include "smc_device.cuh"
#include "smc_nest.h"

int main(int argc, char **argv)
{
    // memo_sparse: the memo evaluated at a pseudo-random subset of the
    // knowledge points (as the kernel's deferred, grouped checks take them),
    // the last one always
    const bool sparse = argc > 1 && strcmp(argv[1], "memo_sparse") == 0;
    const bool use_memo = sparse || (argc > 1 && strcmp(argv[1], "memo") == 0);
    const bool force_nest = use_memo || (argc > 1 && strcmp(argv[1], "nest") == 0);
    int S, NA, NN;
    if (scanf("%d %d %d", &S, &NA, &NN) != 3) return 2;
    std::vector<int32_t> coef((size_t)NA * S), op(NA);
    std::vector<double> bound(NA);
    for (int a = 0; a < NA; ++a) {
        if (scanf("%d %lf", &op[a], &bound[a]) != 2) return 2;
        for (int i = 0; i < S; ++i) if (scanf("%d", &coef[(size_t)a * S + i]) != 1) return 2;
    }
    std::vector<smc_node> nodes(NN);
    for (auto &nd : nodes)
        if (scanf("%d %d %lf %lf", &nd.kind, &nd.arg, &nd.lo, &nd.hi) != 4) return 2;
    std::vector<smc::FNode> tree;
    int root = -1;
    std::string err;
    if (smc::parse_formula(nodes.data(), NN, NA, tree, root, err) != SMC_OK) { printf("parse: %s\n", err.c_str()); return 1; }
    MonProg P;
    NestProg NP;
    std::vector<int> used;
    int rc = force_nest ? SMC_E_UNSUPPORTED : smc::compile_formula(tree, root, NA, INFINITY, P, used, err);
    const bool nest = rc == SMC_E_UNSUPPORTED;
    if (nest) rc = smc::compile_nested(tree, root, NA, 1.0e300, NP, used, err);
    if (rc != SMC_OK) { printf("compile: %s\n", err.c_str()); return 1; }
    const int nu = (int)used.size();
    std::vector<int64_t> thr(2 * (size_t)std::max(nu, 1));
    uint32_t aneg = 0;
    for (int b = 0; b < nu; ++b) {
        bool ng;
        smc::atom_threshold(op[used[b]], bound[used[b]], thr[2 * b], thr[2 * b + 1], ng);
        if (ng) aneg |= 1u << b;
    }
    int n_paths;
    if (scanf("%d", &n_paths) != 1) return 2;
    for (int i = 0; i < n_paths; ++i) {
        int n, closed;
        double tmin;
        if (scanf("%d %d %lf", &n, &closed, &tmin) != 3) return 2;
        std::vector<int32_t> x((size_t)n * S);
        std::vector<double> t(n);
        for (auto &v : x) if (scanf("%d", &v) != 1) return 2;
        for (auto &v : t) if (scanf("%lf", &v) != 1) return 2;
        if (nest) {  // the recorded path: atom bits per state, then what follows it
            std::vector<uint32_t> w(n);
            for (int k = 0; k < n; ++k) {
                uint32_t ab = 0;
                for (int b = 0; b < nu; ++b) {
                    long long L = 0;
                    for (int s = 0; s < S; ++s) L += (long long)coef[(size_t)used[b] * S + s] * x[(size_t)k * S + s];
                    const uint32_t in = (L >= thr[2 * b]) & (L <= thr[2 * b + 1]);
                    ab |= (in ^ ((aneg >> b) & 1u)) << b;
                }
                w[k] = ab;
            }
            const NestTrace T{t.data(), w.data(), 1, (int64_t)n - 1, closed ? 2 : 3, tmin};
            NestVal d = nest_decide(NP, T);
            if (use_memo && n > 0) {
                // garbage in every cell: only zeroing at the record may clear them
                std::vector<uint32_t> memo((size_t)std::max(NP.n_slots, 1) * n, 0xA5A5A5A5u);
                for (int k = 0; k < n; ++k) {
                    for (int sl = 0; sl < NP.n_slots; ++sl) memo[(size_t)sl * n + k] = 0;
                    const bool last = k == n - 1;
                    for (int half = 0; half < 2; ++half) {
                        const uint32_t h = (uint32_t)(i * 2654435761u) ^ (uint32_t)((2 * k + half) * 40503u);
                        if (sparse && !(last && half) && ((h >> 7) % 3u) != 0u) continue;
                        NestTrace U{t.data(), w.data(), 1, k, 0, 0.0, nullptr, 0};
                        if (half) {
                            U.end = last ? (closed ? 2 : 3) : 1;
                            U.tnext = last ? tmin : t[k + 1];
                        }
                        const NestVal a = nest_decide(NP, U);
                        U.memo = memo.data();
                        U.mslot = n;
                        const NestVal b = nest_decide(NP, U);
                        if (a.v != b.v || (a.v && a.d != b.d)) {
                            printf("mismatch path %d q %lld: %d %lld vs %d %lld\n", i, 2ll * k + half, a.v,
                                   (long long)a.d, b.v, (long long)b.d);
                            return 3;
                        }
                        if (last && half) d = b;
                    }
                }
            }
            printf("%d %lld\n", d.v, d.v ? (long long)d.d : -1ll);
            continue;
        }
        // the replay order of the SSA kernels: draw of state k's entry time
        // (when the monitor asks for it), then state k; after the last state
        // the end of the path (closed) or a lower bound on the next entry time
        double tc[SMC_MAX_UNITS * 32];
        MonLane ml;
        int v = 0;
        long long q = -1;
        for (int k = 0; k < n && !v; ++k) {
            if (k > 0) {
                if (ml.pend || __double_as_longlong(t[k]) > ml.hb) v = mon_draw(ml, P, t[k], tc);
                if (v) { q = 2 * (long long)k - 1; break; }
            }
            uint32_t ab = 0;
            for (int b = 0; b < nu; ++b) {
                long long L = 0;
                for (int s = 0; s < S; ++s) L += (long long)coef[(size_t)used[b] * S + s] * x[(size_t)k * S + s];
                const uint32_t in = (L >= thr[2 * b]) & (L <= thr[2 * b + 1]);
                ab |= (in ^ ((aneg >> b) & 1u)) << b;
            }
            ml.ab = ab;
            if (k == 0) mon_start(ml, P);
            v = mon_state(ml, P, t[k], tc);
            if (v) q = 2 * (long long)k;
        }
        if (!v && n > 0) {
            if (closed) v = mon_close(ml, P);
            else v = mon_draw<false>(ml, P, tmin, tc);
            if (v) q = 2 * (long long)n - 1;
        }
        printf("%d %lld\n", v, q);
    }
    return 0;
}
