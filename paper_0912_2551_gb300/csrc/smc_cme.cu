// smc_cme.cu -- exact time-bounded reachability on small networks by
// uniformisation of the CTMC (Sec. 2.2's chain solved numerically instead of
// sampled).  Sec. 5 compares the statistical estimate with PRISM's numerical
// model checking (Fig. 4); this is that comparison's exact side, as a
// validator of smc_estimate on models whose reachable state space fits.
//
// The states reachable from x0 are enumerated breadth first; goal states
// (the property holds there) and failure states (an until's left operand is
// false) are absorbing, and so are states with a count above `cap`
// (truncation: their mass is reported, it bounds the error).  With the
// uniformisation rate L >= every exit rate, P = I + Q / L and
//   P(reach goal by T) = sum_k Poisson(k; L T) goal_mass(pi0 P^k),
// the goal mass being non-decreasing because goal states are absorbing.
// The iterations pi_{k+1} = pi_k P run on the GPU in FP64 (CSR of P^T, one
// thread per state, goal and truncated mass reduced per iteration); the
// Poisson weights come from log-gamma on the host.
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <deque>
#include <string>
#include <unordered_map>
#include <vector>

#include "smc_cme.h"

namespace {

__global__ void cme_step_kernel(int64_t n, const int64_t *rowptr, const int32_t *col, const double *val,
                                const double *x, double *y, const uint8_t *kind, double *mass)
{
    __shared__ double s_goal[8], s_trunc[8];
    double g = 0.0, tr = 0.0;
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x) {
        double acc = 0.0;
        for (int64_t q = rowptr[j]; q < rowptr[j + 1]; ++q) acc = fma(val[q], x[col[q]], acc);
        y[j] = acc;
        if (kind[j] == 1) g += acc;
        else if (kind[j] == 3) tr += acc;
    }
    for (int o = 16; o > 0; o >>= 1) {
        g += __shfl_xor_sync(0xffffffffu, g, o);
        tr += __shfl_xor_sync(0xffffffffu, tr, o);
    }
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) { s_goal[w] = g; s_trunc[w] = tr; }
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0.0, b = 0.0;
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) { a += s_goal[i]; b += s_trunc[i]; }
        atomicAdd(&mass[0], a);
        atomicAdd(&mass[1], b);
    }
}

struct VecHash {
    size_t operator()(const std::vector<int32_t> &v) const
    {
        uint64_t h = 1469598103934665603ull;
        for (int32_t x : v) h = (h ^ (uint32_t)x) * 1099511628211ull;
        return (size_t)h;
    }
};

}  // namespace

namespace smc {

double cme_propensity(const CmeModel &M, int k, const int32_t *x)
{
    int ra = M.reactants[2 * k], rb = M.reactants[2 * k + 1];
    if (ra < 0 && rb >= 0) { ra = rb; rb = -1; }
    int64_t h;
    if (ra < 0) h = 1;
    else if (rb < 0) h = x[ra];
    else if (ra == rb) h = (int64_t)x[ra] * ((int64_t)x[ra] - 1) / 2;
    else h = (int64_t)x[ra] * (int64_t)x[rb];
    double a = M.rates[k] * (double)h;
    for (int q = 0; q < M.n_fact; ++q) {
        if (M.f_reac[q] != k) continue;
        const double xv = (double)x[M.f_spec[q]];
        double xn = xv;
        for (int i = 1; i < M.f_pow[q]; ++i) xn *= xv;
        const double *c = M.f_par + 4 * q;
        a *= (c[0] + c[1] * xn) / (c[2] + c[3] * xn);
    }
    return a;
}

int cme_reach(const CmeModel &M, const CmePredicate &pred, double t_end, int32_t cap, int64_t max_states,
              CmeResult &out, std::string &err, cudaStream_t s)
{
    const int S = M.S, R = M.R;
    // atom bit vector of a state
    auto bits = [&](const int32_t *x) {
        uint32_t ab = 0;
        for (int a = 0; a < pred.n_atoms; ++a) {
            if (pred.expr && pred.expr[a].op >= 0) {
                ab |= (uint32_t)expr_atom_holds(pred.expr[a], x) << a;
                continue;
            }
            int64_t L = 0;
            for (int i = 0; i < S; ++i) L += (int64_t)pred.coef[(size_t)a * S + i] * x[i];
            const uint32_t in = (L >= pred.lo[a]) & (L <= pred.hi[a]);
            ab |= (in ^ (uint32_t)pred.neg[a]) << a;
        }
        return ab;
    };
    // kind: 0 transient, 1 goal, 2 failure, 3 truncated
    std::unordered_map<std::vector<int32_t>, int64_t, VecHash> index;
    std::vector<std::vector<int32_t>> states;
    std::vector<uint8_t> kind;
    std::vector<double> exit;
    struct Edge { int64_t from, to; double rate; };
    std::vector<Edge> edges;
    std::deque<int64_t> queue;
    auto visit = [&](const std::vector<int32_t> &x) -> int64_t {
        auto it = index.find(x);
        if (it != index.end()) return it->second;
        const int64_t id = (int64_t)states.size();
        index.emplace(x, id);
        states.push_back(x);
        const uint32_t ab = bits(x.data());
        uint8_t k = 0;
        if ((pred.goal >> ab) & 1ull) k = 1;
        else if (!((pred.stay >> ab) & 1ull)) k = 2;
        else
            for (int i = 0; i < S; ++i)
                if (x[i] > cap) k = 3;
        kind.push_back(k);
        exit.push_back(0.0);
        if (k == 0) queue.push_back(id);
        return id;
    };
    visit(std::vector<int32_t>(M.x0, M.x0 + S));
    std::vector<int32_t> y(S);
    while (!queue.empty()) {
        const int64_t i = queue.front();
        queue.pop_front();
        for (int k = 0; k < R; ++k) {
            const double a = cme_propensity(M, k, states[i].data());
            if (!(a > 0.0)) continue;
            bool neg = false;
            for (int c = 0; c < S; ++c) {
                y[c] = states[i][c] + M.stoich[(size_t)k * S + c];
                neg = neg || y[c] < 0;
            }
            if (neg) { err = "a reaction with positive propensity drives a count negative"; return -1; }
            const int64_t j = visit(y);
            if ((int64_t)states.size() > max_states) { err = "more reachable states than max_states"; return -4; }
            exit[i] += a;
            if (j != i) edges.push_back({i, j, a});
        }
    }
    const int64_t n = (int64_t)states.size();
    double lam = 0.0;
    for (int64_t i = 0; i < n; ++i) lam = std::max(lam, exit[i]);
    out.n_states = n;
    out.lambda_t = lam * t_end;
    // CSR of P^T: row j holds P_ij for every i with a transition into j,
    // plus the self loop 1 - exit_i / lam
    std::vector<int64_t> cnt(n + 1, 0);
    for (const Edge &e : edges) ++cnt[e.to + 1];
    for (int64_t j = 0; j < n; ++j) ++cnt[j + 1];  // self loop
    for (int64_t j = 0; j < n; ++j) cnt[j + 1] += cnt[j];
    std::vector<int32_t> col(cnt[n]);
    std::vector<double> val(cnt[n]);
    std::vector<int64_t> fill(cnt.begin(), cnt.end() - 1);
    for (int64_t j = 0; j < n; ++j) {
        col[fill[j]] = (int32_t)j;
        val[fill[j]++] = lam > 0.0 ? 1.0 - exit[j] / lam : 1.0;
    }
    for (const Edge &e : edges) {
        col[fill[e.to]] = (int32_t)e.from;
        val[fill[e.to]++] = e.rate / lam;
    }
    // Poisson weights w_k, k = 0..K, K where the right tail is below 1e-14
    const double mu = lam * t_end;
    const int64_t K = (int64_t)std::ceil(mu + 10.0 * std::sqrt(mu) + 30.0);
    // compensated (Neumaier) sums: a plain sum of thousands of weights
    // rounds at ~1e-13, more than the tail it would measure
    struct Sum {
        double s = 0.0, c = 0.0;
        void add(double v)
        {
            const double t = s + v;
            c += std::fabs(s) >= std::fabs(v) ? (s - t) + v : (v - t) + s;
            s = t;
        }
        double value() const { return s + c; }
    };
    // Each weight's exponent -mu + k ln mu - lgamma(k + 1) cancels terms of
    // size ~mu ln mu, so the weights carry a common relative error of about
    // mu ln mu x 2^-53; dividing by their sum removes it (the mass beyond K
    // is below 1e-14).  The tail beyond K is reported from the next terms.
    auto weight = [&](int64_t k) {
        return mu > 0.0 ? std::exp(-mu + (double)k * std::log(mu) - std::lgamma((double)k + 1.0))
                        : (k == 0 ? 1.0 : 0.0);
    };
    std::vector<double> w(K + 1);
    Sum wsum;
    for (int64_t k = 0; k <= K; ++k) {
        w[k] = weight(k);
        wsum.add(w[k]);
    }
    const double norm = wsum.value();
    for (int64_t k = 0; k <= K; ++k) w[k] /= norm;
    // beyond K the terms fall by at least mu / (K + 2) < 1 each step
    out.poisson_tail = mu > 0.0 ? weight(K + 1) / (1.0 - mu / (double)(K + 2)) : 0.0;
    out.iterations = K;
    // device iterations
    int64_t *d_rp = nullptr;
    int32_t *d_col = nullptr;
    double *d_val = nullptr, *d_x = nullptr, *d_y = nullptr, *d_mass = nullptr;
    uint8_t *d_kind = nullptr;
    auto release = [&]() {
        cudaFree(d_rp); cudaFree(d_col); cudaFree(d_val); cudaFree(d_x); cudaFree(d_y); cudaFree(d_mass);
        cudaFree(d_kind);
    };
#define CME_CK(call)                                                              \
    do {                                                                          \
        cudaError_t e_ = (call);                                                  \
        if (e_ != cudaSuccess) {                                                  \
            err = std::string(#call) + ": " + cudaGetErrorString(e_);             \
            release();                                                            \
            return e_ == cudaErrorMemoryAllocation ? -2 : -3;                     \
        }                                                                         \
    } while (0)
    CME_CK(cudaMalloc(&d_rp, (n + 1) * 8));
    CME_CK(cudaMalloc(&d_col, col.size() * 4));
    CME_CK(cudaMalloc(&d_val, val.size() * 8));
    CME_CK(cudaMalloc(&d_x, n * 8));
    CME_CK(cudaMalloc(&d_y, n * 8));
    CME_CK(cudaMalloc(&d_kind, n));
    CME_CK(cudaMalloc(&d_mass, (K + 1) * 2 * 8));
    CME_CK(cudaMemcpyAsync(d_rp, cnt.data(), (n + 1) * 8, cudaMemcpyHostToDevice, s));
    CME_CK(cudaMemcpyAsync(d_col, col.data(), col.size() * 4, cudaMemcpyHostToDevice, s));
    CME_CK(cudaMemcpyAsync(d_val, val.data(), val.size() * 8, cudaMemcpyHostToDevice, s));
    CME_CK(cudaMemcpyAsync(d_kind, kind.data(), n, cudaMemcpyHostToDevice, s));
    CME_CK(cudaMemsetAsync(d_x, 0, n * 8, s));
    CME_CK(cudaMemsetAsync(d_mass, 0, (K + 1) * 2 * 8, s));
    const double one = 1.0;
    CME_CK(cudaMemcpyAsync(d_x, &one, 8, cudaMemcpyHostToDevice, s));  // pi_0 = x0 (state 0)
    const int block = 256;
    const int grid = (int)std::min<int64_t>(1024, (n + block - 1) / block);
    // goal / truncated mass of pi_0
    std::vector<double> mass((K + 1) * 2, 0.0);
    if (kind[0] == 1) mass[0] = 1.0;
    if (kind[0] == 3) mass[1] = 1.0;
    for (int64_t k = 1; k <= K; ++k) {
        cme_step_kernel<<<grid, block, 0, s>>>(n, d_rp, d_col, d_val, d_x, d_y, d_kind, d_mass + 2 * k);
        CME_CK(cudaGetLastError());
        std::swap(d_x, d_y);
    }
    std::vector<double> dm((K + 1) * 2);
    CME_CK(cudaMemcpyAsync(dm.data(), d_mass, dm.size() * 8, cudaMemcpyDeviceToHost, s));
    CME_CK(cudaStreamSynchronize(s));
    release();
#undef CME_CK
    for (int64_t k = 1; k <= K; ++k) { mass[2 * k] = dm[2 * k]; mass[2 * k + 1] = dm[2 * k + 1]; }
    Sum p, tr;
    for (int64_t k = 0; k <= K; ++k) {
        p.add(w[k] * mass[2 * k]);
        tr.add(w[k] * mass[2 * k + 1]);
    }
    out.p = p.value();
    out.truncated = tr.value();
    return 0;
}

}  // namespace smc
