// Batched solves of many independent EDA problems of uneven size (random training splits, class
// subsets): a native host runtime over the single-problem path.
//
// Problems are ordered by an estimated cost, largest first, and taken from one shared queue by
// `workers` host threads. Each worker owns a non-blocking CUDA stream and drives its problems through
// eda_build, block-size tuning, eda_solve; the handles are destroyed after all workers have joined
// (a cudaFree waits for the whole device). The per-problem kernels are small and latency-bound
// (cluster eigensolves on 2-16 SMs, Krylov sweeps over a few MB), so running many problems side by
// side is what fills the GPU. The Krylov loop keeps its host decisions (rank loss, convergence
// checks), which is why concurrency comes from streams and host workers rather than from one
// persistent kernel over a device-side queue.
//
// Block-size tuning: for each problem shape (precision, d, n rounded to 64, k rounded to 16) the first
// problem of that shape times one M-apply of width b on its own handle for the candidate widths and
// keeps the b that minimises (ceil(t / b) + 2) * T(b), the cost of the about t / b + 2 blocks a solve
// of t pairs takes; later problems of the same shape reuse the choice.
#include "eda_internal.cuh"

#include <algorithm>
#include <atomic>
#include <cmath>
#include <map>
#include <mutex>
#include <thread>
#include <tuple>
#include <vector>

namespace eda {
namespace {

using TuneKey = std::tuple<int, int64_t, int64_t, int>;
std::mutex g_tune_mu;
std::map<TuneKey, int> g_tune;

double est_cost(const eda_problem& p) {
    // Gram (d n^2) plus the Krylov sweeps (about 6 sweeps of d (n + k) per block of t / b + 2)
    const double n = (double)p.n, k = (double)p.k, d = (double)p.d;
    return d * n * n + 6.0 * d * (n + k) * ((double)p.t + 16.0);
}

int tune_block(eda_handle h, int t, cudaStream_t s, int* b_out) {
    const int prec = h->cfg.prec;
    const TuneKey key{prec, h->d, (h->n + 63) / 64, (h->k + 15) / 16};
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        auto it = g_tune.find(key);
        if (it != g_tune.end()) {
            *b_out = it->second;
            return EDA_OK;
        }
    }
    const int cand[4] = {4, 8, 16, 32};
    const int bmax = 32;
    const bool f32io = prec == EDA_F32 || prec == EDA_BF16;   // the FP64 solvers (also EDA_F64_TC) take FP64 blocks
    const size_t esz = f32io ? 4 : 8;
    void* buf = nullptr;
    EDA_CUDA_TRY(cudaMalloc(&buf, 2 * (size_t)h->d * bmax * esz));
    char* X = static_cast<char*>(buf);
    char* Y = X + (size_t)h->d * bmax * esz;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    int rc = EDA_OK;
    double best = INFINITY;
    int best_b = 8;
    do {
        if (cudaMemsetAsync(buf, 0, 2 * (size_t)h->d * bmax * esz, s) != cudaSuccess ||
            cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
            rc = EDA_ERR_CUDA;
            break;
        }
        const int io = f32io ? EDA_F32 : EDA_F64;
        for (int b : cand) {
            if (b > std::max(t, 4)) break;
            if ((rc = eda_apply_exp(h, EDA_OP_M, 0.0, X, Y, h->d, b, io, s)) != EDA_OK) break;   // warm-up
            cudaEventRecord(e0, s);
            for (int r = 0; r < 2; ++r)
                if ((rc = eda_apply_exp(h, EDA_OP_M, 0.0, X, Y, h->d, b, io, s)) != EDA_OK) break;
            cudaEventRecord(e1, s);
            if (rc != EDA_OK) break;
            if (cudaEventSynchronize(e1) != cudaSuccess) {
                rc = EDA_ERR_CUDA;
                break;
            }
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            const double cost = (std::ceil((double)t / b) + 2.0) * (ms / 2.0);
            if (cost < best) {
                best = cost;
                best_b = b;
            }
        }
    } while (false);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaStreamSynchronize(s);
    cudaFree(buf);
    if (rc != EDA_OK) return rc;
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        g_tune[key] = best_b;
    }
    *b_out = best_b;
    return EDA_OK;
}

bool valid_problem(const eda_problem& p) {
    return p.X && p.labels && p.V && p.lambda && p.d >= 1 && p.n >= 2 && p.k >= 1 && p.k <= p.n &&
           p.ldx >= p.d && p.t >= 1 && p.t <= p.n + p.k && p.t <= p.d && p.tol > 0.0 &&
           (p.x_dtype == EDA_F64 || p.x_dtype == EDA_F32) && p.block_b >= 0;
}

}  // namespace
}  // namespace eda

using namespace eda;

extern "C" int eda_solve_batched(eda_problem* probs, int32_t nprob, const eda_config* cfg, int32_t workers,
                                 void* stream) {
    if (nprob < 0 || (nprob > 0 && !probs)) return EDA_ERR_INVALID_ARG;
    eda_config c;
    if (cfg) c = *cfg;
    else eda_config_default(&c);
    for (int i = 0; i < nprob; ++i)
        if (!valid_problem(probs[i])) return EDA_ERR_INVALID_ARG;
    if (nprob == 0) return EDA_OK;
    const bool autotune = c.block_b <= 0;
    if (autotune) c.block_b = 8;   // build-time value; the tuned width is set before the solve

    int dev = 0;
    EDA_CUDA_TRY(cudaGetDevice(&dev));
    cudaStream_t caller = static_cast<cudaStream_t>(stream);
    cudaEvent_t start = nullptr;
    EDA_CUDA_TRY(cudaEventCreateWithFlags(&start, cudaEventDisableTiming));
    EDA_CUDA_TRY(cudaEventRecord(start, caller));

    std::vector<int> order(nprob);
    for (int i = 0; i < nprob; ++i) order[i] = i;
    std::stable_sort(order.begin(), order.end(),
                     [&](int a, int b) { return est_cost(probs[a]) > est_cost(probs[b]); });
    const int W = std::max(1, std::min<int>(workers > 0 ? workers : 16, nprob));
    std::vector<eda_handle> handles(nprob, nullptr);
    std::vector<cudaStream_t> streams(W, nullptr);
    std::vector<cudaEvent_t> done(W, nullptr);
    std::atomic<int> next{0};
    std::vector<int> worker_rc(W, EDA_OK);

    auto work = [&](int w) {
        symeig_set_shared_gpu(true);   // no grid-wide barriers while other problems run beside this one
        if (cudaSetDevice(dev) != cudaSuccess ||
            cudaStreamCreateWithFlags(&streams[w], cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&done[w], cudaEventDisableTiming) != cudaSuccess ||
            cudaStreamWaitEvent(streams[w], start, 0) != cudaSuccess) {
            worker_rc[w] = EDA_ERR_CUDA;
            return;
        }
        cudaStream_t s = streams[w];
        for (int q = next++; q < nprob; q = next++) {
            eda_problem& p = probs[order[q]];
            eda_config pc = c;
            if (p.block_b > 0) pc.block_b = p.block_b;
            // the one-pass bf16 exp-apply is a cooperative launch with grid-wide barriers: like the eigensolver's
            // cooperative grid, it is kept off threads whose problems share the GPU with others
            pc.tc_fused = -1;
            eda_handle h = nullptr;
            int rc = eda_build(p.X, p.x_dtype, p.d, p.n, p.ldx, p.labels, p.k, &pc, s, &h);
            handles[order[q]] = h;
            if (rc == EDA_OK && autotune && p.block_b <= 0) {
                int b = 8;
                rc = tune_block(h, p.t, s, &b);
                if (rc == EDA_OK) h->cfg.block_b = b;
            }
            if (rc == EDA_OK) {
                p.info.relres = nullptr;
                rc = eda_solve(h, p.t, p.tol, nullptr, 0, p.V, p.lambda, nullptr, &p.info, s);
            }
            p.status = rc;
        }
        cudaEventRecord(done[w], s);
    };
    std::vector<std::thread> pool;
    pool.reserve(W);
    for (int w = 0; w < W; ++w) pool.emplace_back(work, w);
    for (auto& th : pool) th.join();

    int rc = EDA_OK;
    for (int w = 0; w < W; ++w) {
        if (worker_rc[w] != EDA_OK && rc == EDA_OK) rc = worker_rc[w];
        if (done[w]) cudaStreamWaitEvent(caller, done[w], 0);
    }
    for (int w = 0; w < W; ++w) {
        if (streams[w]) cudaStreamSynchronize(streams[w]);
    }
    for (eda_handle h : handles)
        if (h) eda_destroy(h);
    for (int w = 0; w < W; ++w) {
        if (done[w]) cudaEventDestroy(done[w]);
        if (streams[w]) cudaStreamDestroy(streams[w]);
    }
    cudaEventDestroy(start);
    for (int i = 0; i < nprob && rc == EDA_OK; ++i) {
        const int st = probs[order[i]].status;
        if (st != EDA_OK && st != EDA_ERR_NOT_CONVERGED) rc = st;
    }
    if (rc == EDA_OK) {
        for (int i = 0; i < nprob; ++i)
            if (probs[i].status == EDA_ERR_NOT_CONVERGED) rc = EDA_ERR_NOT_CONVERGED;
    }
    return rc;
}
