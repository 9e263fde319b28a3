// C ABI: handle lifetime, the build step (Section 1 and Algorithm 2 steps 1-4 in Gram/eigen
// form), exp-vector products (Theorem 3.1, Algorithm 2 steps 6L-12L) and projection.
#include "eda_internal.cuh"

#include <algorithm>
#include <cfloat>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

namespace eda {

namespace {
thread_local int g_last_cuda_error = 0;
thread_local char g_last_cuda_msg[256] = "no error";
std::atomic<uint64_t> g_launches{0};
}  // namespace

void note_cuda_error(cudaError_t e, const char* file, int line) {
    g_last_cuda_error = (int)e;
    const char* base = file ? std::strrchr(file, '/') : nullptr;
    base = base ? base + 1 : (file ? file : "?");
    std::snprintf(g_last_cuda_msg, sizeof(g_last_cuda_msg), "%s (%s:%d)", cudaGetErrorString(e), base, line);
}

int ensure_workspace(eda_ctx* h, size_t bytes) {
    if (h->ws_bytes >= bytes) return EDA_OK;
    if (h->ws) {
        EDA_CUDA_TRY(cudaFree(h->ws));
        h->ws = nullptr;
        h->ws_bytes = 0;
    }
    void* p = nullptr;
    EDA_CUDA_TRY(cudaMalloc(&p, bytes));
    h->ws = p;
    h->ws_bytes = bytes;
    return EDA_OK;
}
std::atomic<uint64_t>& launch_counter() { return g_launches; }

// Solve-side entry points implemented in lanczos.cu.
int solve_impl(eda_ctx* h, int t, double tol, const double* V0, int b0, double* V, double* lambda, double* Y,
               eda_solve_info* info, cudaStream_t s);
int m_apply(eda_ctx* h, int b, const double* X, int64_t ldx, double* Y, int64_t ldy, double* tmp, double* P,
            double* Q, double* partial, size_t partial_cap, cudaStream_t s);
int m_apply_f32(eda_ctx* h, int b, const float* X, int64_t ldx, float* Y, int64_t ldy, float* tmp, double* P,
                double* Q, double* partial, size_t partial_cap, cudaStream_t s);
int arnoldi_impl(eda_ctx* h, int t, double tol, double* Vout, double* lambda, eda_solve_info* info, cudaStream_t s);
int direct_impl(eda_ctx* h, int t, double* Vout, double* lambda, eda_solve_info* info, cudaStream_t s);

namespace {
// B (k x n) = A^T for A (n x k), both column-major.
__global__ void k_transpose_nk(int n, int k, const double* __restrict__ A, double* __restrict__ B) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (int64_t)n * k) return;
    const int i = (int)(e % n), j = (int)(e / n);
    B[(int64_t)i * k + j] = A[e];
}
}  // namespace

// Cross Grams G_WB = H_W^T H_B and G_BW = G_WB^T for the composed FP64 M-apply (the mixed-precision
// refinement, the FP64 Krylov phase with m_form = 1, and the FP64 verification after refills);
// formed once per handle. part: split-K partials of at least n k doubles.
int ensure_cross_gram(eda_ctx* h, double* part, size_t pcap, cudaStream_t s) {
    if (h->GWB) return EDA_OK;
    const int n = (int)h->n, k = h->k;
    const size_t xb = ((size_t)n * k * 8 + 255) & ~size_t(255);
    void* xp = nullptr;
    EDA_CUDA_TRY(cudaMalloc(&xp, 2 * xb));
    h->xblock = xp;
    h->GWB = static_cast<double*>(xp);
    h->GBW = reinterpret_cast<double*>(static_cast<char*>(xp) + xb);
    EDA_TRY(gemm_tn_f64(h->d, n, k, 1.0, h->HW, h->d, h->HB, h->d, 0.0, h->GWB, n, part, pcap, s));
    k_transpose_nk<<<ceil_div((int64_t)n * k, 256), 256, 0, s>>>(n, k, h->GWB, h->GBW);
    EDA_LAUNCHED();
    return EDA_OK;
}

namespace {

constexpr int kEigClusterMaxN = 512;   // the eigensolver's cluster path (no grid barrier) up to this size
constexpr double kSigRel = 32.0;   // eigenvalues <= kSigRel * n * eps * lambda_max are the Gram's null space
constexpr int kLanczosSteps = 64;  // steps of the largest-eigenvalue Lanczos run on a Gram
constexpr double kLmaxAccept = 8.0;  // accept its theta_1 when its residual is <= kLmaxAccept * eps * theta_1
constexpr int kLanczosStepsLarge = 64;    // the same run on a large Gram (n >= kOzSmallMinN, tensor-core mode)
constexpr int64_t kTcMinMiDefault = 4;    // EDA_F64_TC: tensor-core products from d (n + k) >= 4 x 2^20 on

size_t align256(size_t b) { return (b + 255) & ~size_t(255); }

int tc_operands(eda_ctx* h, cudaStream_t s);
int tc_grams(eda_ctx* h, cudaStream_t s);

int read_status(eda_ctx* h, cudaStream_t s, int* out) {
    EDA_CUDA_TRY(cudaMemcpyAsync(out, h->status, sizeof(int), cudaMemcpyDeviceToHost, s));
    EDA_CUDA_TRY(cudaStreamSynchronize(s));
    return EDA_OK;
}

int status_to_code(int st) {
    if (st & ST_TIMEOUT) return EDA_ERR_TIMEOUT;
    if (st & ST_NONFINITE) return EDA_ERR_NONFINITE;
    if (st & (ST_BADLABEL | ST_EMPTYCLASS)) return EDA_ERR_BAD_LABELS;
    return EDA_OK;
}

// Allocate the handle's device block: factors, Grams, eigenpairs, operators, status, barrier.
int alloc_handle(eda_ctx* h, bool with_labels) {
    const size_t d = h->d, n = h->n, k = h->k;
    const size_t N = std::max(n, k);
    size_t bytes = 0;
    auto add = [&](size_t b) { bytes += align256(b); };
    add(d * (n + k) * 8);     // [HW HB]
    if (with_labels) {
        add(k * 4);           // counts
        add((k + 1) * 4);     // offsets
        add(n * 4);           // perm
        add(k * d * 8);       // mu_j
        add(d * 8);           // mu
    }
    add(n * n * 8);           // GW
    add(k * k * 8);           // GB
    add(n * 8);               // evals_w
    add(k * 8);               // evals_b
    add(n * n * 8);           // evecs_w
    add(k * k * 8);           // evecs_b
    add(n * n * 8);           // KW
    add(k * k * 8);           // KB
    add(256);                 // status
    add(256);                 // barrier
    // build scratch: eigensolver workspace + gram partials + phi/Newton-Schulz temporaries
    const size_t pcap = std::max<size_t>(1u << 19, N * N);
    add(symeig_work_bytes((int)N, (int)N));
    add(pcap * 8);
    add(3 * N * N * 8 + 256);
    // the second, concurrent Gram eigensolve: its workspace, partials and temporaries
    add(symeig_work_bytes((int)std::min(n, k), (int)std::min(n, k)));
    add(std::max<size_t>(1u << 16, std::min(n, k) * std::min(n, k)) * 8);
    add(3 * std::min(n, k) * std::min(n, k) * 8 + 256);
    // the Lanczos / scaling-and-squaring build of small Grams: partials of the second stream, the two
    // Lanczos workspaces and results, the squaring work of both Grams
    add(std::max<size_t>(1u << 17, 64 * k * k) * 8);
    add(symeig_work_bytes((int)n, 1));
    add(symeig_work_bytes((int)k, 1));
    add(8 * 8);
    add(6 * n * n * 8);
    add(6 * k * k * 8);
    add(4096);
    h->block_bytes = bytes + 4096;
    void* p = nullptr;
    EDA_CUDA_TRY(cudaMalloc(&p, h->block_bytes));
    h->block = p;
    Arena a{static_cast<char*>(p), h->block_bytes, 0};
    h->HW = a.take<double>(d * (n + k));
    h->HB = h->HW + d * n;
    if (with_labels) {
        h->counts = a.take<int32_t>(k);
        h->offsets = a.take<int32_t>(k + 1);
        h->perm = a.take<int32_t>(n);
        h->mu_j = a.take<double>(k * d);
        h->mu = a.take<double>(d);
    }
    h->GW = a.take<double>(n * n);
    h->GB = a.take<double>(k * k);
    h->evals_w = a.take<double>(n);
    h->evals_b = a.take<double>(k);
    h->evecs_w = a.take<double>(n * n);
    h->evecs_b = a.take<double>(k * k);
    h->KW = a.take<double>(n * n);
    h->KB = a.take<double>(k * k);
    h->status = a.take<int>(64);
    unsigned* bar = a.take<unsigned>(64);
    h->bar = GridBarrier{bar, bar + 32, h->cfg.wait_limit > 0 ? (long long)h->cfg.wait_limit : kGridSpinDefault};
    h->build_arena_off = a.used;
    if (!h->KB || !bar) return EDA_ERR_OOM;
    EDA_CUDA_TRY(cudaMemset(h->status, 0, 256));
    EDA_CUDA_TRY(cudaMemset(bar, 0, 256));
    return EDA_OK;
}

// Eigenpairs of one Gram G (m x m): all eigenvalues, vectors for the significant ones, and
// K(alpha). Returns lambda_max and the number of significant eigenpairs.
// The part of a Gram eigensolve after its eigenvalues are on the host (w, ascending): lambda_max, the
// significant eigenpairs (above kSigRel * m * eps * lambda_max) and their vectors, refined by one
// Newton-Schulz step. tmp: 3 m^2 + 64 doubles; part/pcap: split-K partials.
int gram_eigen_finish(eda_ctx* h, int m, const std::vector<double>& w, double* evals, double* evecs,
                      SymEigWork* ws, double* tmp, double* part, size_t pcap, double* lmax, int* nsig, int* first_out,
                      cudaStream_t s) {
    for (double v : w)
        if (!std::isfinite(v)) return EDA_ERR_NONFINITE;
    *lmax = std::max(w[m - 1], 0.0);
    const double thr = kSigRel * m * DBL_EPSILON * *lmax;
    int first = 0;
    while (first < m && !(w[first] > thr)) ++first;
    *nsig = m - first;
    *first_out = first;
    if (*nsig > 0) {
        EDA_TRY(symeig_vectors(m, *nsig, evals + first, evecs, m, ws, h->cfg.seed, 1e-7, s));
        EDA_TRY(newton_schulz_f64(m, *nsig, evecs, m, 1, tmp, part, pcap, s));
    }
    return EDA_OK;
}

int gram_eigen(eda_ctx* h, int m, double* G, double* evals, double* evecs, Arena& scratch, double* part, size_t pcap,
               double* lmax, int* nsig, cudaStream_t s) {
    if (m <= 0) {
        *lmax = 0.0;
        *nsig = 0;
        return EDA_OK;
    }
    SymEigWork ws{};
    EDA_TRY(symeig_work_carve(scratch, m, m, h->bar, &ws));
    EDA_TRY(symeig_values(m, G, m, 0, m - 1, evals, &ws, h->status, s));
    std::vector<double> w(m);
    EDA_CUDA_TRY(cudaMemcpyAsync(w.data(), evals, m * sizeof(double), cudaMemcpyDeviceToHost, s));
    EDA_CUDA_TRY(cudaStreamSynchronize(s));
    int st = 0;
    EDA_TRY(read_status(h, s, &st));
    if (int c = status_to_code(st)) return c;
    double* tmp = scratch.take<double>(3 * (size_t)m * m + 64);
    if (!tmp) return EDA_ERR_OOM;
    int first = 0;
    EDA_TRY(gram_eigen_finish(h, m, w, evals, evecs, &ws, tmp, part, pcap, lmax, nsig, &first, s));
    h->nsig_first = first;   // only meaningful for the last call; the callers store their own copy
    return EDA_OK;
}

// Both Gram eigensolves side by side on two streams (each runs in one thread-block cluster, so
// together they still leave most SMs idle): eigenvalues of G_W on s and of G_B on a second stream,
// one host wait for both, then the eigenvectors of each on its stream. Separate workspaces,
// temporaries and split-K partials per solve; the second stream joins s before returning.
int gram_eigen_pair(eda_ctx* h, Arena& scratch, double* partW, size_t pcapW, int* nsw, int* nsb, int* first_w,
                    int* first_b, cudaStream_t s) {
    const int n = (int)h->n, k = h->k;
    SymEigWork wsW{}, wsB{};
    EDA_TRY(symeig_work_carve(scratch, n, n, h->bar, &wsW));
    EDA_TRY(symeig_work_carve(scratch, k, k, h->bar, &wsB));
    const size_t pcapB = std::max<size_t>(1u << 16, (size_t)k * k);
    double* partB = scratch.take<double>(pcapB);
    double* tmpW = scratch.take<double>(3 * (size_t)n * n + 64);
    double* tmpB = scratch.take<double>(3 * (size_t)k * k + 64);
    if (!partB || !tmpW || !tmpB) return EDA_ERR_OOM;
    cudaStream_t s2 = nullptr;
    cudaEvent_t fork = nullptr, join = nullptr;
    int rc = EDA_OK;
    std::vector<double> ww(n), wb(k);
    do {
        if (cudaStreamCreateWithFlags(&s2, cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&fork, cudaEventDisableTiming) != cudaSuccess ||
            cudaEventCreateWithFlags(&join, cudaEventDisableTiming) != cudaSuccess ||
            cudaEventRecord(fork, s) != cudaSuccess || cudaStreamWaitEvent(s2, fork, 0) != cudaSuccess) {
            rc = EDA_ERR_CUDA;
            break;
        }
        // two reductions in flight at once: both on the cluster path (a cooperative grid needs every SM it
        // spans, and the two would share the handle's grid-barrier words)
        const bool prev_shared = symeig_set_shared_gpu(true);
        rc = symeig_values(n, h->GW, n, 0, n - 1, h->evals_w, &wsW, h->status, s);
        if (rc == EDA_OK) rc = symeig_values(k, h->GB, k, 0, k - 1, h->evals_b, &wsB, h->status, s2);
        symeig_set_shared_gpu(prev_shared);
        if (rc != EDA_OK) break;
        if (cudaMemcpyAsync(ww.data(), h->evals_w, n * sizeof(double), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
            cudaMemcpyAsync(wb.data(), h->evals_b, k * sizeof(double), cudaMemcpyDeviceToHost, s2) != cudaSuccess ||
            cudaStreamSynchronize(s2) != cudaSuccess) {
            rc = EDA_ERR_CUDA;
            break;
        }
        int st = 0;
        if ((rc = read_status(h, s, &st)) != EDA_OK) break;
        if ((rc = status_to_code(st)) != EDA_OK) break;
        if ((rc = gram_eigen_finish(h, n, ww, h->evals_w, h->evecs_w, &wsW, tmpW, partW, pcapW, &h->lmax_w, nsw,
                                    first_w, s)) != EDA_OK)
            break;
        if ((rc = gram_eigen_finish(h, k, wb, h->evals_b, h->evecs_b, &wsB, tmpB, partB, pcapB, &h->lmax_b, nsb,
                                    first_b, s2)) != EDA_OK)
            break;
    } while (false);
    if (s2) {
        if (join && cudaEventRecord(join, s2) == cudaSuccess) cudaStreamWaitEvent(s, join, 0);
        else cudaStreamSynchronize(s2);
        cudaStreamDestroy(s2);   // released once its queued work has finished
    }
    if (fork) cudaEventDestroy(fork);
    if (join) cudaEventDestroy(join);
    return rc;
}


// A second stream for the independent halves of the build (the two Grams), joined back into the
// caller's stream when it goes out of scope.
struct AuxStream {
    cudaStream_t main = nullptr, aux = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    int open(cudaStream_t s) {
        main = s;
        if (cudaStreamCreateWithFlags(&aux, cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&ev_fork, cudaEventDisableTiming) != cudaSuccess ||
            cudaEventCreateWithFlags(&ev_join, cudaEventDisableTiming) != cudaSuccess)
            return EDA_ERR_CUDA;
        return EDA_OK;
    }
    int fork() {
        EDA_CUDA_TRY(cudaEventRecord(ev_fork, main));
        EDA_CUDA_TRY(cudaStreamWaitEvent(aux, ev_fork, 0));
        return EDA_OK;
    }
    int join() {
        EDA_CUDA_TRY(cudaEventRecord(ev_join, aux));
        EDA_CUDA_TRY(cudaStreamWaitEvent(main, ev_join, 0));
        return EDA_OK;
    }
    ~AuxStream() {
        if (aux) {
            if (!ev_join || cudaEventRecord(ev_join, aux) != cudaSuccess ||
                cudaStreamWaitEvent(main, ev_join, 0) != cudaSuccess)
                cudaStreamSynchronize(aux);
            cudaStreamDestroy(aux);   // released once its queued work has finished
        }
        if (ev_fork) cudaEventDestroy(ev_fork);
        if (ev_join) cudaEventDestroy(ev_join);
    }
};

// lambda_max of a Gram from its Lanczos run (theta_1, theta_2, |z_m|, beta_m), or -1 when theta_1 is not
// accepted. The residual r = beta_m |z_m| of the top Ritz pair bounds the distance from theta_1 to an
// eigenvalue of G; theta_1 is accepted only when r <= kLmaxAccept * eps * theta_1, i.e. when the pair is
// converged to working precision. That the eigenvalue within r is the largest one (and not one below a
// top eigenvalue the run never found) rests on the random start block, as for any Krylov eigensolver;
// no gap estimate enters (the Ritz gap theta_1 - theta_2 can exceed the true gap, so a quadratic bound
// built on it would not be a bound). A rejected run falls back to the symmetric eigensolver.
double lmax_accepted(const double* o) {
    const double t1 = o[0], r = o[2] * o[3];
    if (!std::isfinite(t1) || !std::isfinite(r)) return -1.0;
    if (!(r <= kLmaxAccept * DBL_EPSILON * std::max(t1, 0.0))) return -1.0;
    return std::max(t1, 0.0);
}

// lambda_max of one Gram (m x m) by a Lanczos run of kLanczosStepsLarge steps. Its top Ritz value theta_1
// with residual bound r is taken when r <= kLmaxAccept eps theta_1. Otherwise, when theta_1 + r < below
// (the other Gram's lambda_max, which then sets c^2), theta_1 is kept as the estimate and theta_1 + r as
// an upper bound (for the squaring's scale); else the full eigensolver's largest eigenvalue (into w) is
// taken. *lmax: the value, *lbound: an upper bound for the squaring (equal to *lmax when exact).
int gram_lmax_one(eda_ctx* h, int m, const double* G, double* w, Arena& scratch, double below, double* lmax,
                  double* lbound, cudaStream_t s) {
    SymEigWork ws{};
    EDA_TRY(symeig_work_carve(scratch, m, 1, h->bar, &ws));
    double* out = scratch.take<double>(4);
    if (!out) return EDA_ERR_OOM;
    EDA_TRY(lanczos_top(m, G, m, std::min(m, kLanczosStepsLarge), h->cfg.seed, &ws, out, s));
    double o[4];
    EDA_CUDA_TRY(cudaMemcpyAsync(o, out, sizeof(o), cudaMemcpyDeviceToHost, s));
    EDA_CUDA_TRY(cudaStreamSynchronize(s));
    double l = lmax_accepted(o);
    const double r = o[2] * o[3];
    if (l < 0.0 && std::isfinite(o[0]) && std::isfinite(r) && o[0] + r < below) {
        *lmax = std::max(o[0], 0.0);
        *lbound = std::max(o[0] + r, 0.0);
        return EDA_OK;
    }
    if (l < 0.0) {
        EDA_TRY(symeig_values(m, G, m, m - 1, m - 1, w, &ws, h->status, s));
        double top = 0.0;
        EDA_CUDA_TRY(cudaMemcpyAsync(&top, w, sizeof(double), cudaMemcpyDeviceToHost, s));
        EDA_CUDA_TRY(cudaStreamSynchronize(s));
        int st = 0;
        EDA_TRY(read_status(h, s, &st));
        if (int c = status_to_code(st)) return c;
        if (!std::isfinite(top)) return EDA_ERR_NONFINITE;
        l = std::max(top, 0.0);
    }
    *lmax = l;
    *lbound = l;
    return EDA_OK;
}

// lambda_max of G_W and G_B without their eigenvectors: one Lanczos run per Gram, side by side on two
// streams (aux is already forked from s and holds the G_B product), one host wait for both; a Gram
// whose residual does not accept its estimate falls back to the full eigensolver's largest eigenvalue.
int gram_lmax_pair(eda_ctx* h, Arena& scratch, AuxStream& aux, cudaStream_t s) {
    const int n = (int)h->n, k = h->k;
    SymEigWork wsW{}, wsB{};
    EDA_TRY(symeig_work_carve(scratch, n, 1, h->bar, &wsW));
    EDA_TRY(symeig_work_carve(scratch, k, 1, h->bar, &wsB));
    double* out = scratch.take<double>(8);
    if (!out) return EDA_ERR_OOM;
    EDA_TRY(lanczos_top(n, h->GW, n, std::min(n, kLanczosSteps), h->cfg.seed, &wsW, out, s));
    EDA_TRY(lanczos_top(k, h->GB, k, std::min(k, kLanczosSteps), h->cfg.seed, &wsB, out + 4, aux.aux));
    EDA_TRY(aux.join());
    double o[8];
    EDA_CUDA_TRY(cudaMemcpyAsync(o, out, sizeof(o), cudaMemcpyDeviceToHost, s));
    EDA_CUDA_TRY(cudaStreamSynchronize(s));
    double lw = lmax_accepted(o), lb = lmax_accepted(o + 4);
    for (int g = 0; g < 2; ++g) {
        double& l = g == 0 ? lw : lb;
        if (l >= 0.0) continue;
        const int m = g == 0 ? n : k;
        double* w = g == 0 ? h->evals_w : h->evals_b;
        EDA_TRY(symeig_values(m, g == 0 ? h->GW : h->GB, m, m - 1, m - 1, w, g == 0 ? &wsW : &wsB, h->status, s));
        double top = 0.0;
        EDA_CUDA_TRY(cudaMemcpyAsync(&top, w, sizeof(double), cudaMemcpyDeviceToHost, s));
        EDA_CUDA_TRY(cudaStreamSynchronize(s));
        int st = 0;
        EDA_TRY(read_status(h, s, &st));
        if (int c = status_to_code(st)) return c;
        if (!std::isfinite(top)) return EDA_ERR_NONFINITE;
        l = std::max(top, 0.0);
    }
    h->lmax_w = lw;
    h->lmax_b = lb;
    return EDA_OK;
}

// The Grams' eigenpairs (eigenvalues, significant eigenvectors) for a handle whose K came from
// scaling and squaring: computed on first request (exported eigenvalues, K(alpha) for another alpha).
// lambda_max and c^2 keep the values the build used.
int ensure_eigen(eda_ctx* h, cudaStream_t s) {
    if (h->eig_ready) return EDA_OK;
    const int n = (int)h->n, k = h->k;
    const size_t N = std::max<int64_t>(n, k);
    Arena scratch{static_cast<char*>(h->block), h->block_bytes, h->build_arena_off};
    const size_t pcap = std::max<size_t>(1u << 19, N * N);
    double* part = scratch.take<double>(pcap);
    if (!part) return EDA_ERR_OOM;
    const size_t mark = scratch.used;
    double lm = 0.0;
    int ns = 0;
    EDA_TRY(gram_eigen(h, n, h->GW, h->evals_w, h->evecs_w, scratch, part, pcap, &lm, &ns, s));
    h->nsig_w = ns;
    scratch.used = mark;
    EDA_TRY(gram_eigen(h, k, h->GB, h->evals_b, h->evecs_b, scratch, part, pcap, &lm, &ns, s));
    h->nsig_b = ns;
    h->eig_ready = true;
    return EDA_OK;
}

// Everything after H_W, H_B exist: Grams, eigenpairs, c^2, K operators, and for the mixed
// solver single-precision copies of the factors.
int finish_build(eda_ctx* h, cudaStream_t s) {
    const int n = (int)h->n, k = h->k;
    const int64_t d = h->d;
    if (h->cfg.prec == EDA_F32) {
        const size_t bw = align256((size_t)d * n * sizeof(float)), bb = align256((size_t)d * k * sizeof(float));
        void* p = nullptr;
        EDA_CUDA_TRY(cudaMalloc(&p, bw + bb));
        h->block32 = p;
        h->HW32 = static_cast<float*>(p);
        h->HB32 = reinterpret_cast<float*>(static_cast<char*>(p) + bw);
        EDA_TRY((copy_mat<double, float>(d, n, h->HW, d, h->HW32, d, s)));
        EDA_TRY((copy_mat<double, float>(d, k, h->HB, d, h->HB32, d, s)));
    }
    Arena scratch{static_cast<char*>(h->block), h->block_bytes, h->build_arena_off};
    const size_t N = std::max<int64_t>(n, k);
    const size_t pcap = std::max<size_t>(1u << 19, N * N);
    double* part = scratch.take<double>(pcap);
    if (!part) return EDA_ERR_OOM;
    // Small Grams: lambda_max by Lanczos and K by scaling and squaring (dense products that fill the
    // GPU) instead of the eigensolver's sequential column steps; the eigenpairs follow on request.
    // The B half (G_B, its Lanczos run, its K, the cross Gram) runs on a second stream beside the W half.
    const bool by_squaring = n <= kLanczosMaxN && k <= kLanczosMaxN;
    const bool cross = h->cfg.prec == EDA_F32 || h->cfg.prec == EDA_BF16 || h->cfg.prec == EDA_F64_TC ||
                       h->cfg.m_form == 1;
    AuxStream aux;
    double* partB = nullptr;
    size_t pcapB = 0;
    // the tensor-core products from a size of Z on (tc_min_mi), the FP64 ones below it
    const int64_t zmi = h->cfg.tc_min_mi == 0 ? kTcMinMiDefault : h->cfg.tc_min_mi;
    const bool tc = h->cfg.prec == EDA_F64_TC && (zmi < 0 || d * (int64_t)(n + k) >= (zmi << 20));
    // Large G_W in tensor-core mode: lambda_max by Lanczos and K_W by scaling and squaring with
    // FP64-accurate tensor-core products, instead of the n-step tridiagonalisation and the
    // back-transformation of the eigensolver; G_B keeps its route.
    const bool sq_w_tc = tc && !by_squaring && n >= kOzSmallMinN;
    if (sq_w_tc) {
        // four n x n split operands: the squaring's two factors, then K_W and G_W for the solves
        const size_t b1 = align256(oz_operand_bytes(n, n));
        void* p = nullptr;
        EDA_CUDA_TRY(cudaMalloc(&p, 4 * b1));
        h->ozsmall = p;
    }
    if (tc) {
        // every Gram as a block of Z^T Z on the tensor cores, from the split Z the sweeps use as well
        EDA_TRY(tc_operands(h, s));
        EDA_TRY(tc_grams(h, s));
        EDA_TRY(check_finite_f64(n, n, h->GW, n, h->status, s));
        EDA_TRY(check_finite_f64(k, k, h->GB, k, h->status, s));
        if (by_squaring) {
            EDA_TRY(aux.open(s));
            pcapB = std::max<size_t>(1u << 17, 64 * (size_t)k * k);
            partB = scratch.take<double>(pcapB);
            if (!partB) return EDA_ERR_OOM;
            EDA_TRY(aux.fork());
        }
    } else if (by_squaring) {
        EDA_TRY(aux.open(s));
        pcapB = std::max<size_t>(1u << 17, 64 * (size_t)k * k);
        partB = scratch.take<double>(pcapB);
        if (!partB) return EDA_ERR_OOM;
        EDA_TRY(aux.fork());
        {
            // algorithmic work of the SYRK G_W = H_W^T H_W: d n (n + 1) flops (one triangle), reading H_W once
            ProfScope prof("gram", s, (double)d * n * (n + 1.0), 8.0 * (double)d * n);
            EDA_TRY(syrk_f64(d, n, 1.0, h->HW, d, 0.0, h->GW, n, part, pcap, s));
        }
        EDA_TRY(syrk_f64(d, k, 1.0, h->HB, d, 0.0, h->GB, k, partB, pcapB, aux.aux));
        EDA_TRY(check_finite_f64(n, n, h->GW, n, h->status, s));
        EDA_TRY(check_finite_f64(k, k, h->GB, k, h->status, aux.aux));
    } else {
        {
            ProfScope prof("gram", s, (double)d * ((double)n * (n + 1.0) + (double)k * (k + 1.0)),
                           8.0 * (double)d * (n + k));
            EDA_TRY(syrk_f64(d, n, 1.0, h->HW, d, 0.0, h->GW, n, part, pcap, s));
            EDA_TRY(syrk_f64(d, k, 1.0, h->HB, d, 0.0, h->GB, k, part, pcap, s));
        }
        EDA_TRY(check_finite_f64(n, n, h->GW, n, h->status, s));
        EDA_TRY(check_finite_f64(k, k, h->GB, k, h->status, s));
    }
    const size_t mark = scratch.used;
    int nsw = 0, nsb = 0, first_w = 0, first_b = 0;
    double lbound_w = 0.0;   // the large-G_W route: an upper bound of lambda_max(G_W) for the squaring
    if (by_squaring) {
        EDA_TRY(gram_lmax_pair(h, scratch, aux, s));
    } else if (sq_w_tc) {
        EDA_TRY(gram_eigen(h, k, h->GB, h->evals_b, h->evecs_b, scratch, part, pcap, &h->lmax_b, &nsb, s));
        first_b = h->nsig_first;
        scratch.used = mark;
        const double below = h->cfg.c2 > 0.0 ? DBL_MAX : h->lmax_b;   // with a given c^2 nothing is compared
        EDA_TRY(gram_lmax_one(h, n, h->GW, h->evals_w, scratch, below, &h->lmax_w, &lbound_w, s));
    } else if (n <= kEigClusterMaxN && k <= kEigClusterMaxN) {
        // both on the cluster path (no grid barrier): solve side by side
        EDA_TRY(gram_eigen_pair(h, scratch, part, pcap, &nsw, &nsb, &first_w, &first_b, s));
    } else {
        EDA_TRY(gram_eigen(h, n, h->GW, h->evals_w, h->evecs_w, scratch, part, pcap, &h->lmax_w, &nsw, s));
        first_w = h->nsig_first;
        scratch.used = mark;
        EDA_TRY(gram_eigen(h, k, h->GB, h->evals_b, h->evecs_b, scratch, part, pcap, &h->lmax_b, &nsb, s));
        first_b = h->nsig_first;
    }
    scratch.used = mark;
    h->nsig_w = nsw;
    h->nsig_b = nsb;
    h->eig_ready = !by_squaring && !sq_w_tc;
    h->lmax_w_bound = sq_w_tc ? std::max(lbound_w, h->lmax_w) : h->lmax_w;
    if (h->cfg.c2 > 0.0) {
        h->c2 = h->cfg.c2;
    } else {
        const double m = std::max(h->lmax_w, h->lmax_b);
        if (!(m > 0.0)) return EDA_ERR_INVALID_ARG;   // both scatter matrices vanish
        h->c2 = h->cfg.tau / m;
    }
    if (by_squaring) {
        double* workW = scratch.take<double>(6 * (size_t)n * n);
        double* workB = scratch.take<double>(6 * (size_t)k * k);
        if (!workW || !workB) return EDA_ERR_OOM;
        {
            ProfScope prof("phi_squaring", s);
            EDA_TRY(aux.fork());
            EDA_TRY(phi_by_squaring(n, h->GW, -0.5 * h->c2, h->lmax_w, h->KW, workW, s));
            EDA_TRY(phi_by_squaring(k, h->GB, h->c2, h->lmax_b, h->KB, workB, aux.aux));
            if (cross) EDA_TRY(ensure_cross_gram(h, partB, pcapB, aux.aux));
            EDA_TRY(aux.join());
        }
        scratch.used = mark;
    } else {
        double* tmp = scratch.take<double>(N * N + 64);
        if (!tmp) return EDA_ERR_OOM;
        if (sq_w_tc) {
            double* workW = scratch.take<double>(6 * (size_t)n * n);
            if (!workW) return EDA_ERR_OOM;
            ProfScope prof("phi_squaring", s);
            const size_t b1 = align256(oz_operand_bytes(n, n));
            const OzSquare oz{h->ozsmall, static_cast<char*>(h->ozsmall) + b1, h->status};
            EDA_TRY(phi_by_squaring(n, h->GW, -0.5 * h->c2, h->lmax_w_bound, h->KW, workW, s, &oz));
        } else {
            EDA_TRY(phi_operator(n, nsw, h->evals_w + first_w, h->evecs_w, n, -0.5 * h->c2, h->KW, tmp, s));
        }
        EDA_TRY(phi_operator(k, nsb, h->evals_b + first_b, h->evecs_b, k, h->c2, h->KB, tmp, s));
    }
    if (cross && !by_squaring) EDA_TRY(ensure_cross_gram(h, part, pcap, s));
    if (sq_w_tc) {
        // K_W and G_W are symmetric: column i is row i, so the column-scaled split serves as the left factor
        const size_t b1 = align256(oz_operand_bytes(n, n));
        char* p = static_cast<char*>(h->ozsmall);
        EDA_TRY(oz_operand_make(h->KW, n, n, n, true, p + 2 * b1, &h->ozKW, h->status, s));
        EDA_TRY(oz_operand_make(h->GW, n, n, n, true, p + 3 * b1, &h->ozGW, h->status, s));
    }
    if (h->cfg.prec == EDA_BF16) {
        // bf16 H_W, H_B tiled for sweep 1, bf16 H K tiled for sweep 2, and the staging
        // buffers of X and P with their tensor maps (zeroed: padded rows are read as zeros)
        const int64_t ldh = tc_pad_rows(d);
        const int ldq = std::max(tc_pad_cols(n), tc_pad_cols(k));
        const size_t sz[7] = {align256((size_t)tc_tiles_sweep1(d, n) * 2), align256((size_t)tc_tiles_sweep2(d, n) * 2),
                              align256((size_t)tc_tiles_sweep1(d, k) * 2), align256((size_t)tc_tiles_sweep2(d, k) * 2),
                              align256((size_t)ldh * 32 * 2) * 2, align256((size_t)ldq * 32 * 2) * 2,
                              align256(tc_partial_floats(std::max(n, k)) * 4)};
        size_t tot = 0;
        for (size_t v : sz) tot += v;
        void* p = nullptr;
        EDA_CUDA_TRY(cudaMalloc(&p, tot));
        h->block32 = p;
        EDA_CUDA_TRY(cudaMemsetAsync(p, 0, tot, s));
        char* c = static_cast<char*>(p);
        auto bf = [&](size_t off) { return reinterpret_cast<__nv_bfloat16*>(c + off); };
        size_t off = 0;
        __nv_bfloat16* HcW = bf(off); off += sz[0];
        __nv_bfloat16* HKW = bf(off); off += sz[1];
        __nv_bfloat16* HcB = bf(off); off += sz[2];
        __nv_bfloat16* HKB = bf(off); off += sz[3];
        __nv_bfloat16* Xhi = bf(off);
        __nv_bfloat16* Xlo = bf(off + sz[4] / 2); off += sz[4];
        __nv_bfloat16* Qhi = bf(off);
        __nv_bfloat16* Qlo = bf(off + sz[5] / 2); off += sz[5];
        float* partial = reinterpret_cast<float*>(c + off); off += sz[6];
        EDA_TRY(tc_factor_make(h->HW, d, n, h->KW, HcW, HKW, &h->tcW, h->status, s));
        EDA_TRY(tc_factor_make(h->HB, d, k, h->KB, HcB, HKB, &h->tcB, h->status, s));
        EDA_TRY(tc_buffers_make(ldh, ldq, Xhi, Xlo, Qhi, Qlo, partial, tc_partial_floats(std::max(n, k)), &h->tcbuf));
        // the one-pass form for both factors (decided together: the M-apply chains them) when the larger fits
        if (h->cfg.tc_fused >= 0 && tc_fused_grid(d, std::max(n, k)) > 0) {
            const size_t fz[4] = {align256((size_t)tc_fused_elems(d, n) * 2), align256((size_t)tc_fused_elems(d, k) * 2),
                                  align256(tc_fused_partial_floats(d, std::max(n, k)) * 4), 256};
            void* fp = nullptr;
            EDA_CUDA_TRY(cudaMalloc(&fp, fz[0] + fz[1] + fz[2] + fz[3]));
            h->fblock = fp;
            char* fc = static_cast<char*>(fp);
            EDA_CUDA_TRY(cudaMemsetAsync(fc + fz[0] + fz[1] + fz[2], 0, fz[3], s));   // grid-barrier words
            EDA_TRY(tc_fused_make(h->HW, d, n, h->KW, -0.5 * h->c2, reinterpret_cast<__nv_bfloat16*>(fc), &h->tcW,
                                  h->status, s));
            EDA_TRY(tc_fused_make(h->HB, d, k, h->KB, h->c2, reinterpret_cast<__nv_bfloat16*>(fc + fz[0]), &h->tcB,
                                  h->status, s));
            h->tcbuf.fpartial = reinterpret_cast<float*>(fc + fz[0] + fz[1]);
            h->tcbuf.fbar = reinterpret_cast<unsigned*>(fc + fz[0] + fz[1] + fz[2]);
            h->tcbuf.fspin = h->bar.spin_limit;
        }
    }
    int st = 0;
    EDA_TRY(read_status(h, s, &st));
    return status_to_code(st);
}

// prec = EDA_F64_TC: Z = [H_W H_B] (d x (n + k), one allocation) split into bf16 digit planes twice, scaled
// per column for Z^T Y and per row for Z U, and the narrow staging sized for both reduction lengths.
int tc_operands(eda_ctx* h, cudaStream_t s) {
    const int64_t d = h->d;
    const int nk = (int)h->n + h->k;
    const size_t bT = align256(oz_operand_bytes(nk, d)), bN = align256(oz_operand_bytes(d, nk));
    const size_t bS = align256(oz_narrow_bytes(std::max<int64_t>(d, nk), sm_count(), nk));
    void* p = nullptr;
    EDA_CUDA_TRY(cudaMalloc(&p, bT + bN + bS));
    h->ozblock = p;
    char* c = static_cast<char*>(p);
    EDA_TRY(oz_operand_make(h->HW, d, nk, d, true, c, &h->ozT, h->status, s));
    EDA_TRY(oz_operand_make(h->HW, d, d, nk, false, c + bT, &h->ozN, h->status, s));
    EDA_TRY(oz_narrow_make(std::max<int64_t>(d, nk), sm_count(), nk, c + bT + bN, &h->oznb));
    return EDA_OK;
}

// prec = EDA_F64_TC: the Grams G_W, G_B and the cross Grams G_WB, G_BW as the blocks of Z^T Z, computed with
// the FP64-accurate tensor-core product of the split Z with itself in one launch (the blocks meeting the
// upper triangle, the rest mirrored). A column of Z has the same scale and digits on either side, so
// Z^T Z comes out exactly symmetric.
int tc_grams(eda_ctx* h, cudaStream_t s) {
    const int64_t d = h->d;
    const int n = (int)h->n, k = h->k, nk = n + k;
    ProfScope prof("gram", s, (double)d * nk * (nk + 1.0), 8.0 * (double)d * nk);
    double* GZ = nullptr;
    EDA_CUDA_TRY(cudaMalloc(&GZ, (size_t)nk * nk * 8));
    int rc = oz_gemm_tiled(h->ozT, h->ozT, 1.0, 0.0, nullptr, 0, GZ, nk, true, h->status, s);
    if (rc == EDA_OK && !h->GWB) {
        const size_t xb = ((size_t)n * k * 8 + 255) & ~size_t(255);
        void* xp = nullptr;
        if (cudaMalloc(&xp, 2 * xb) != cudaSuccess) {
            cudaGetLastError();
            rc = EDA_ERR_OOM;
        } else {
            h->xblock = xp;
            h->GWB = static_cast<double*>(xp);
            h->GBW = reinterpret_cast<double*>(static_cast<char*>(xp) + xb);
        }
    }
    if (rc == EDA_OK) rc = copy_mat_f64(n, n, GZ, nk, h->GW, n, s);
    if (rc == EDA_OK) rc = copy_mat_f64(k, k, GZ + (size_t)n * nk + n, nk, h->GB, k, s);
    if (rc == EDA_OK) rc = copy_mat_f64(n, k, GZ + (size_t)n * nk, nk, h->GWB, n, s);
    if (rc == EDA_OK) rc = copy_mat_f64(k, n, GZ + n, nk, h->GBW, k, s);
    cudaStreamSynchronize(s);   // GZ is released below
    cudaFree(GZ);
    return rc;
}

bool valid_cfg(const eda_config& c) {
    return c.block_b >= 1 && c.check_every >= 1 && (c.c2 > 0.0 || c.tau > 0.0) &&
           (c.prec == EDA_F64 || c.prec == EDA_F32 || c.prec == EDA_BF16 || c.prec == EDA_F64_TC) &&
           (c.m_form == 0 || c.m_form == 1);
}

}  // namespace
}  // namespace eda

using namespace eda;

extern "C" {

int eda_config_default(eda_config* cfg) {
    if (!cfg) return EDA_ERR_INVALID_ARG;
    std::memset(cfg, 0, sizeof(*cfg));
    cfg->prec = EDA_F64;
    cfg->block_b = 8;
    cfg->m_max = 0;
    cfg->check_every = 1;
    cfg->tau = 10.0;
    cfg->c2 = 0.0;
    cfg->seed = 1;
    cfg->true_residuals = 0;
    return EDA_OK;
}

int eda_build(const void* X, int32_t x_dtype, int64_t d, int64_t n, int64_t ldx, const int32_t* labels, int32_t k,
              const eda_config* cfg, void* stream, eda_handle* out) {
    if (!out || !X || !labels || d < 1 || n < 2 || k < 1 || k > n || ldx < d || n > (1 << 20) || k > 12288)
        return EDA_ERR_INVALID_ARG;
    if (x_dtype != EDA_F64 && x_dtype != EDA_F32) return EDA_ERR_INVALID_ARG;
    eda_config c;
    if (cfg) c = *cfg;
    else eda_config_default(&c);
    if (!valid_cfg(c)) return EDA_ERR_INVALID_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    eda_ctx* h = new (std::nothrow) eda_ctx();
    if (!h) return EDA_ERR_OOM;
    h->d = d;
    h->n = n;
    h->k = k;
    h->cfg = c;
    int rc = alloc_handle(h, true);
    if (rc == EDA_OK) rc = segment_labels(labels, (int)n, k, h->counts, h->offsets, h->perm, h->status, s);
    if (rc == EDA_OK) {
        int st = 0;
        rc = read_status(h, s, &st);
        if (rc == EDA_OK) rc = status_to_code(st);
    }
    if (rc == EDA_OK)
        rc = build_factors(X, x_dtype, d, (int)n, ldx, k, labels, h->counts, h->offsets, h->perm, h->mu_j, h->mu,
                           h->HW, h->HB, h->status, s);
    if (rc == EDA_OK) {
        int st = 0;
        rc = read_status(h, s, &st);
        if (rc == EDA_OK) rc = status_to_code(st);
    }
    if (rc == EDA_OK) rc = finish_build(h, s);
    if (rc != EDA_OK) {
        eda_destroy(h);
        return rc;
    }
    *out = h;
    return EDA_OK;
}

int eda_build_from_factors(const double* HW, int64_t n, const double* HB, int64_t kb, int64_t d,
                           const eda_config* cfg, void* stream, eda_handle* out) {
    if (!out || !HW || !HB || d < 1 || n < 1 || kb < 1 || n > (1 << 20) || kb > (1 << 20)) return EDA_ERR_INVALID_ARG;
    eda_config c;
    if (cfg) c = *cfg;
    else eda_config_default(&c);
    if (!valid_cfg(c)) return EDA_ERR_INVALID_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    eda_ctx* h = new (std::nothrow) eda_ctx();
    if (!h) return EDA_ERR_OOM;
    h->d = d;
    h->n = n;
    h->k = (int32_t)kb;
    h->cfg = c;
    int rc = alloc_handle(h, false);
    if (rc == EDA_OK) rc = copy_mat_f64(d, (int)n, HW, d, h->HW, d, s);
    if (rc == EDA_OK) rc = copy_mat_f64(d, (int)kb, HB, d, h->HB, d, s);
    if (rc == EDA_OK) rc = check_finite_f64(d, (int)n, h->HW, d, h->status, s);
    if (rc == EDA_OK) rc = check_finite_f64(d, (int)kb, h->HB, d, h->status, s);
    if (rc == EDA_OK) rc = finish_build(h, s);
    if (rc != EDA_OK) {
        eda_destroy(h);
        return rc;
    }
    *out = h;
    return EDA_OK;
}

int eda_apply_exp(eda_handle h, int32_t op, double alpha, const void* X, void* Y, int64_t ldx, int32_t b,
                  int32_t io_dtype, void* stream) {
    if (!h || !X || !Y || b < 1 || ldx < h->d) return EDA_ERR_INVALID_ARG;
    if (io_dtype != EDA_F64 && !(io_dtype == EDA_F32 && (h->cfg.prec == EDA_F32 || h->cfg.prec == EDA_BF16)))
        return EDA_ERR_INVALID_ARG;
    const size_t esz = io_dtype == EDA_F64 ? sizeof(double) : sizeof(float);
    if (op != EDA_OP_SW && op != EDA_OP_SB && op != EDA_OP_M && op != EDA_OP_N) return EDA_ERR_INVALID_ARG;
    if (op == EDA_OP_N && io_dtype != EDA_F64) return EDA_ERR_INVALID_ARG;
    const char* xb = static_cast<const char*>(X);
    const char* yb = static_cast<const char*>(Y);
    const size_t span = ((size_t)(b - 1) * ldx + h->d) * esz;
    if (xb < yb + span && yb < xb + span) return EDA_ERR_INVALID_ARG;   // X and Y overlap
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int64_t d = h->d;
    // temporaries: P, Q ((n + k) x b: also the coordinates of the composed M-apply), split-K
    // partials, and one d x b block for op M
    const int N = (int)(h->n + h->k);
    const size_t pcap = std::max<size_t>(1u << 19, (size_t)N * b);
    const size_t need = align256((size_t)N * b * 8) * 2 + align256(pcap * 8) + align256((size_t)d * b * 8) + 4096;
    EDA_TRY(eda::ensure_workspace(h, need));
    Arena a{static_cast<char*>(h->ws), h->ws_bytes, 0};
    double* P = a.take<double>((size_t)N * b);
    double* Q = a.take<double>((size_t)N * b);
    double* part = a.take<double>(pcap);
    double* tmp = a.take<double>((size_t)d * b);
    const double* x = static_cast<const double*>(X);
    double* y = static_cast<double*>(Y);
    if (io_dtype == EDA_F32) {
        const float* xf = static_cast<const float*>(X);
        float* yf = static_cast<float*>(Y);
        if (op == EDA_OP_M) return m_apply_f32(h, b, xf, ldx, yf, ldx, reinterpret_cast<float*>(tmp), P, Q, part, pcap, s);
        const bool isW = (op == EDA_OP_SW);
        const int m = isW ? (int)h->n : h->k;
        const double* K = isW ? h->KW : h->KB;
        if (alpha != (isW ? -0.5 * h->c2 : h->c2)) return EDA_ERR_INVALID_ARG;   // stored operators only
        if (h->cfg.prec == EDA_BF16)
            return exp_apply_tc(isW ? h->tcW : h->tcB, h->tcbuf, isW ? "exp_apply_w" : "exp_apply_b", b, xf, ldx, yf,
                                ldx, 0, h->status, s);
        return exp_apply<float>(d, isW ? h->HW32 : h->HB32, K, m, isW ? "exp_apply_w" : "exp_apply_b", b, xf, ldx, yf,
                                ldx, P, Q, part, pcap, s);
    }
    if (op == EDA_OP_M) return m_apply(h, b, x, ldx, y, ldx, tmp, P, Q, part, pcap, s);
    if (op == EDA_OP_N) {
        EDA_TRY(ensure_n_operators(h, s));
        // ensure_n_operators may have grown the workspace: take the temporaries again
        EDA_TRY(eda::ensure_workspace(h, need));
        Arena a2{static_cast<char*>(h->ws), h->ws_bytes, 0};
        double* P2 = a2.take<double>((size_t)N * b);
        double* Q2 = a2.take<double>((size_t)N * b);
        double* part2 = a2.take<double>(pcap);
        return n_apply_composed(h, b, x, ldx, y, ldx, P2, Q2, nullptr, part2, pcap, s);
    }
    // K(alpha) for the requested alpha: rebuild from the stored eigenpairs when alpha differs
    const bool isW = (op == EDA_OP_SW);
    const int m = isW ? (int)h->n : h->k;
    const double stored = isW ? -0.5 * h->c2 : h->c2;
    const double* K = isW ? h->KW : h->KB;
    if (alpha != stored) {
        EDA_TRY(ensure_eigen(h, s));
        if (!h->kblock) {
            void* kb = nullptr;
            EDA_CUDA_TRY(cudaMalloc(&kb, 2 * align256((size_t)N * N * 8)));
            h->kblock = kb;
            h->Kalpha = static_cast<double*>(kb);
            h->Kalpha_tmp = reinterpret_cast<double*>(static_cast<char*>(kb) + align256((size_t)N * N * 8));
        }
        double* Kx = h->Kalpha;
        double* t2 = h->Kalpha_tmp;
        const int ns = isW ? h->nsig_w : h->nsig_b;
        const double* lam = (isW ? h->evals_w : h->evals_b) + (m - ns);
        EDA_TRY(phi_operator(m, ns, lam, isW ? h->evecs_w : h->evecs_b, m, alpha, Kx, t2, s));
        K = Kx;
    }
    ExpOp eo{isW ? h->HW : h->HB, K, m, isW ? "exp_apply_w" : "exp_apply_b"};
    return exp_apply_f64(d, eo, b, x, ldx, y, ldx, P, Q, part, pcap, s);
}

int eda_solve(eda_handle h, int32_t t, double tol, const double* V0, int32_t b0, double* V, double* lambda, double* Y,
              eda_solve_info* info, void* stream) {
    if (!h || !V || !lambda || t < 1 || !(tol > 0.0) || (V0 && b0 < 1)) return EDA_ERR_INVALID_ARG;
    return solve_impl(h, t, tol, V0, b0, V, lambda, Y, info, static_cast<cudaStream_t>(stream));
}

int eda_solve_arnoldi(eda_handle h, int32_t t, double tol, double* V, double* lambda, eda_solve_info* info,
                      void* stream) {
    if (!h || !V || !lambda || t < 1 || !(tol > 0.0)) return EDA_ERR_INVALID_ARG;
    if (h->cfg.prec != EDA_F64 && h->cfg.prec != EDA_F64_TC) return EDA_ERR_INVALID_ARG;
    return arnoldi_impl(h, t, tol, V, lambda, info, static_cast<cudaStream_t>(stream));
}

int eda_solve_direct(eda_handle h, int32_t t, double* V, double* lambda, eda_solve_info* info, void* stream) {
    if (!h || !V || !lambda || t < 1) return EDA_ERR_INVALID_ARG;
    if (h->cfg.prec != EDA_F64 && h->cfg.prec != EDA_F64_TC) return EDA_ERR_INVALID_ARG;
    return direct_impl(h, t, V, lambda, info, static_cast<cudaStream_t>(stream));
}

int eda_project(eda_handle h, const double* V, int32_t t, const void* Xq, int32_t xq_dtype, int64_t m, int64_t ldq,
                double* P, void* stream) {
    if (!h || !V || !Xq || !P || t < 1 || m < 0 || ldq < h->d) return EDA_ERR_INVALID_ARG;
    if (xq_dtype != EDA_F64) return EDA_ERR_INVALID_ARG;
    if (m == 0) return EDA_OK;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const size_t pcap = std::max<size_t>(1u << 19, (size_t)t * m);
    const double* X = static_cast<const double*>(Xq);
    if (h->cfg.prec == EDA_F64_TC && h->ozblock && m <= (int64_t)INT32_MAX) {
        // both factors split (columns of V and of Xq over the d pixels), one tensor-core launch
        const size_t bv = align256(oz_operand_bytes(t, h->d)), bx = align256(oz_operand_bytes(m, h->d));
        EDA_TRY(eda::ensure_workspace(h, align256(pcap * 8) * 4 + bv + bx + 4096));
        char* w = static_cast<char*>(h->ws);
        double* part = reinterpret_cast<double*>(w);
        OzOperand ov, ox;
        EDA_TRY(oz_operand_make(V, h->d, t, h->d, true, w + align256(pcap * 8) * 4, &ov, h->status, s));
        EDA_TRY(oz_operand_make(X, ldq, m, h->d, true, w + align256(pcap * 8) * 4 + bv, &ox, h->status, s));
        return oz_gemm_tiled(ov, ox, 1.0, 0.0, nullptr, 0, P, t, false, h->status, s, part, pcap * 4);
    }
    EDA_TRY(eda::ensure_workspace(h, align256(pcap * 8) + 4096));
    double* part = static_cast<double*>(h->ws);
    return gemm_tn_f64(h->d, t, (int)m, 1.0, V, h->d, X, ldq, 0.0, P, t, part, pcap, s);
}

int eda_get_factors(eda_handle h, double* HW, double* HB, int32_t* counts, int32_t* perm, double* GW, double* GB,
                    double* KW, double* KB, double* evals_w, double* evals_b, void* stream) {
    if (!h) return EDA_ERR_INVALID_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const size_t d = h->d, n = h->n, k = h->k;
    auto cp = [&](void* dst, const void* src, size_t bytes) -> int {
        if (!dst) return EDA_OK;
        if (!src) return EDA_ERR_INVALID_ARG;
        EDA_CUDA_TRY(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToDevice, s));
        return EDA_OK;
    };
    EDA_TRY(cp(HW, h->HW, d * n * 8));
    EDA_TRY(cp(HB, h->HB, d * k * 8));
    EDA_TRY(cp(counts, h->counts, k * 4));
    EDA_TRY(cp(perm, h->perm, n * 4));
    EDA_TRY(cp(GW, h->GW, n * n * 8));
    EDA_TRY(cp(GB, h->GB, k * k * 8));
    EDA_TRY(cp(KW, h->KW, n * n * 8));
    EDA_TRY(cp(KB, h->KB, k * k * 8));
    if (evals_w || evals_b) EDA_TRY(eda::ensure_eigen(h, s));
    EDA_TRY(cp(evals_w, h->evals_w, n * 8));
    EDA_TRY(cp(evals_b, h->evals_b, k * 8));
    return EDA_OK;
}

int eda_get_dims(eda_handle h, int64_t* d, int64_t* n, int32_t* k, double* c2, double* lmax_w, double* lmax_b) {
    if (!h) return EDA_ERR_INVALID_ARG;
    if (d) *d = h->d;
    if (n) *n = h->n;
    if (k) *k = h->k;
    if (c2) *c2 = h->c2;
    if (lmax_w) *lmax_w = h->lmax_w;
    if (lmax_b) *lmax_b = h->lmax_b;
    return EDA_OK;
}

void eda_destroy(eda_handle h) {
    if (!h) return;
    if (h->ws) cudaFree(h->ws);
    if (h->kblock) cudaFree(h->kblock);
    if (h->xblock) cudaFree(h->xblock);
    if (h->ozblock) cudaFree(h->ozblock);
    if (h->ozsmall) cudaFree(h->ozsmall);
    if (h->nblock) cudaFree(h->nblock);
    if (h->block32) cudaFree(h->block32);
    if (h->fblock) cudaFree(h->fblock);
    if (h->block) cudaFree(h->block);
    delete h;
}

const char* eda_strerror(int status) {
    switch (status) {
        case EDA_OK: return "success";
        case EDA_ERR_INVALID_ARG: return "invalid argument";
        case EDA_ERR_BAD_LABELS: return "label outside [0, k) or empty class";
        case EDA_ERR_NONFINITE: return "non-finite value in input or intermediate";
        case EDA_ERR_OOM: return "device allocation failed";
        case EDA_ERR_CUDA: return "CUDA error (see eda_last_cuda_error)";
        case EDA_ERR_TIMEOUT: return "bounded device wait gave up";
        case EDA_ERR_BREAKDOWN: return "Krylov block lost rank and could not be refilled";
        case EDA_ERR_NOT_CONVERGED: return "not converged within the basis limit";
        default: return "unknown status";
    }
}

int eda_last_cuda_error(void) { return g_last_cuda_error; }
const char* eda_last_cuda_error_string(void) { return g_last_cuda_error ? g_last_cuda_msg : "no error"; }
uint64_t eda_kernel_launches(void) { return g_launches.load(); }

}  // extern "C"
