// batched.cu -- many independent problems in one call (gp2s_lml_batched).
//
// The paper's training loop evaluates one LML per MCMC block (App. D); a batch of independent,
// unevenly sized problems (different N, d, radii and bumps) is served here by a pool of worker
// threads, each owning an engine context with its own CUDA stream and workspace.  Problems are
// handed out largest-first from a shared counter, so the streams stay busy and the small problems
// fill the gaps the large ones leave; every problem runs the same kernels as a single gp2s_lml
// call (assembly, multi-RHS CG with FP64 refinement, SLQ), which is what the parity tests cover.
// The worker contexts persist in the parent context, so repeated batched calls reuse their
// workspaces without new allocations once the largest problem has been seen.
//
// Autotuner: problems fall into shape classes (kernel family, d, floor(log2 n)).  Per class it
// tries each launch configuration once on the first problems of that class (block-Jacobi block
// of 64 or 128 rows x CUDA-graph replay of the CG iteration runs on or off), scoring each by the
// problem's wall time per point, and then runs the class on the best one.  The table persists in
// the parent context, so later calls start tuned.  A configuration only changes the block size
// (reported per problem in gp2s_lml_info.bj_block, with the configuration index in
// batch_config); graph replay gives bit-identical results to eager launches.
// GP2S_BATCH_TUNE=0 runs every problem on the defaults.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cstdlib>
#include <cstring>
#include <limits>
#include <mutex>
#include <string>
#include <numeric>
#include <thread>
#include <vector>

#include "gp2s_internal.cuh"

namespace gp2s {

gp2s_status lml_single(gp2s_ctx *c, int64_t n, const double *X, const double *y, const gp2s_hyper *h,
                       const gp2s_opts *o, double *lml, double *grad, gp2s_lml_info *info);   // capi.cu

namespace {

struct BatchConfig {
    int bj_block;   // 64 or 128
    bool graphs;
};
constexpr BatchConfig kBatchConfigs[] = {{64, false}, {128, false}, {64, true}, {128, true}};
constexpr int kNumBatchConfigs = sizeof(kBatchConfigs) / sizeof(kBatchConfigs[0]);

int shape_class(const gp2s_hyper &h, int64_t n)
{
    int lg = 0;
    while ((int64_t(1) << (lg + 1)) <= n) ++lg;
    return (h.family * 8 + h.d) * 64 + lg;
}

}  // namespace

gp2s_status batched_lml(gp2s_ctx *c, int32_t B, const int64_t *n, const double *const *X,
                        const double *const *y, const gp2s_hyper *hyper, const gp2s_opts *opts,
                        double *lml_host, gp2s_lml_info *info_host)
{
    if (B < 0) return set_err(c, GP2S_EINVAL, "B must be >= 0");
    if (B == 0) return GP2S_OK;
    if (!n || !X || !y || !hyper || !lml_host) return set_err(c, GP2S_EINVAL, "batched: NULL argument");
    gp2s_opts o;
    if (opts) o = *opts;
    else gp2s_opts_default(&o);
    // a batch of mid-sized problems is served by SLQ unless the exact path is asked for explicitly
    if (o.logdet == GP2S_LOGDET_AUTO) o.logdet = GP2S_LOGDET_SLQ;
    // device inputs may have been produced on the caller's stream: let that work finish first
    GP2S_CUDA(c, cudaSetDevice(c->device));
    GP2S_CUDA(c, cudaStreamSynchronize(c->stream));

    // worker contexts (created once, kept in the parent)
    const int nworkers = std::max(1, std::min<int>(B, (int)c->batch_workers_max));
    while ((int)c->workers.size() < nworkers) {
        cudaStream_t s = nullptr;
        GP2S_CUDA(c, cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
        gp2s_ctx *w = nullptr;
        gp2s_status st = gp2s_create(&w, c->device, s);
        if (st != GP2S_OK) {
            cudaStreamDestroy(s);
            return set_err(c, st, "batched: cannot create a worker context");
        }
        w->mem_limit = c->mem_limit;
        // graphs per problem are the autotuner's choice (many host threads capturing at once can
        // cost more than the launches they save on small problems)
        w->use_graphs = false;
        c->workers.push_back(w);
        c->worker_streams.push_back(s);
    }
    // largest problems first
    std::vector<int32_t> order(B);
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(), [&](int32_t a, int32_t b) { return n[a] > n[b]; });
    std::atomic<int32_t> next{0};
    std::mutex mu;
    gp2s_status first = GP2S_OK;
    std::string first_msg;
    const char *tune_env = std::getenv("GP2S_BATCH_TUNE");
    const bool tune = !(tune_env && std::strcmp(tune_env, "0") == 0) && o.precision == GP2S_PREC_MIXED &&
                      o.precond == 2 && o.bj_block == 0;
    auto pick = [&](int cls) -> int {
        std::lock_guard<std::mutex> lk(c->tune_mu);
        auto &t = c->tune[cls];
        if (t.count.empty()) {
            t.count.assign(kNumBatchConfigs, 0);
            t.score.assign(kNumBatchConfigs, 0.0);
            t.issued.assign(kNumBatchConfigs, 0);
        }
        if (t.chosen >= 0) return t.chosen;
        for (int k = 0; k < kNumBatchConfigs; ++k)
            if (t.issued[k] == 0) {       // every configuration gets one problem first
                t.issued[k] = 1;
                return k;
            }
        // the best mean time per point so far; final once every configuration has been measured
        int best = 0, measured = 0;
        double bs = 1e300;
        for (int k = 0; k < kNumBatchConfigs; ++k)
            if (t.count[k] > 0) {
                ++measured;
                if (t.score[k] / t.count[k] < bs) {
                    bs = t.score[k] / t.count[k];
                    best = k;
                }
            }
        if (measured == kNumBatchConfigs) t.chosen = best;
        return best;
    };
    auto record = [&](int cls, int k, double sec_per_point) {
        std::lock_guard<std::mutex> lk(c->tune_mu);
        auto &t = c->tune[cls];
        t.score[k] += sec_per_point;
        t.count[k] += 1;
    };
    auto work = [&](int wi) {
        gp2s_ctx *w = c->workers[wi];
        for (;;) {
            const int32_t k = next.fetch_add(1);
            if (k >= B) break;
            const int32_t b = order[k];
            gp2s_lml_info info;
            double v = 0.0;
            gp2s_opts ob = o;
            int cfg = -1, cls = 0;
            if (tune) {
                cls = shape_class(hyper[b], n[b]);
                cfg = pick(cls);
                ob.bj_block = kBatchConfigs[cfg].bj_block;
                w->use_graphs = kBatchConfigs[cfg].graphs;
            } else {
                w->use_graphs = false;
            }
            const auto t0 = std::chrono::steady_clock::now();
            gp2s_status st = lml_single(w, n[b], X[b], y[b], &hyper[b], &ob, &v, nullptr, &info);
            const double sec = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
            if (tune && st == GP2S_OK) record(cls, cfg, sec / (double)std::max<int64_t>(1, n[b]));
            info.batch_config = cfg;
            lml_host[b] = st == GP2S_OK ? v : std::numeric_limits<double>::quiet_NaN();
            if (info_host) {
                if (st == GP2S_OK) info_host[b] = info;
                else std::memset(&info_host[b], 0, sizeof(gp2s_lml_info));
            }
            if (st != GP2S_OK) {
                std::lock_guard<std::mutex> lk(mu);
                if (first == GP2S_OK) {
                    first = st;
                    first_msg = "problem " + std::to_string(b) + ": " + w->err;
                }
            }
        }
    };
    std::vector<std::thread> th;
    for (int wi = 1; wi < nworkers; ++wi) th.emplace_back(work, wi);
    work(0);
    for (auto &t : th) t.join();
    if (first != GP2S_OK) return set_err(c, first, first_msg);
    return GP2S_OK;
}

}  // namespace gp2s
