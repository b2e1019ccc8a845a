// mcmc.cu -- block Metropolis-Hastings training of the hyperparameters (Sec. 4.6, App. D): per
// iteration every block of parameters takes one normal random-walk proposal, rejected outright
// outside the flat prior's bounds and otherwise accepted with probability min(1, exp(LML' - LML)).
// Every proposal costs one LML evaluation on this context; blocks that leave r alone (bump
// centers, radii, amplitudes, sigma2) reuse the last assembly's pattern, so only the values are
// recomputed (opts.pattern_cache = 0).  The state can be written to a checkpoint file and a later
// call resumes from it.
//
// Random numbers: the caller may pass the standard normals (iters x P) and the acceptance
// uniforms (iters x nblocks).  Without them the driver draws its own from a counter-based
// SplitMix64 stream (Vigna's published generator): uniform u = (z >> 11) 2^-53 of
// z = splitmix64(seed ^ (tag << 56 | counter)), normals by Box-Muller from two such uniforms.
#include <cerrno>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "gp2s_internal.cuh"

namespace gp2s {

gp2s_status lml_single(gp2s_ctx *c, int64_t n, const double *X, const double *y, const gp2s_hyper *h,
                       const gp2s_opts *o, double *lml, double *grad, gp2s_lml_info *info);   // capi.cu

namespace {

uint64_t mix64(uint64_t x)
{
    uint64_t z = x + 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// uniform in (0, 1): never exactly 0, so log u is finite
double unit_uniform(uint64_t seed, uint64_t tag, uint64_t counter)
{
    const uint64_t z = mix64(seed ^ ((tag << 56) | (counter & 0x00FFFFFFFFFFFFFFull)));
    return ((double)(z >> 11) + 0.5) * 0x1.0p-53;
}

double std_normal(uint64_t seed, uint64_t counter)
{
    const double u1 = unit_uniform(seed, 1, 2 * counter), u2 = unit_uniform(seed, 1, 2 * counter + 1);
    return std::sqrt(-2.0 * std::log(u1)) * std::cos(2.0 * M_PI * u2);
}

// theta of either family: [centers, radii, amps, (G, ell, w0,) r, sigma2]
gp2s_hyper hyper_from(const gp2s_hyper &h0, const std::vector<double> &th)
{
    gp2s_hyper h = h0;
    const int L = h0.L, d = h0.d;
    h.centers = th.data();
    h.radii = th.data() + L * d;
    h.amps = th.data() + L * d + L;
    const int P = (int)th.size();
    if (h0.family == GP2S_KERNEL_WENDCONV) {
        h.G = th.data() + L * d + 2 * L;
        h.ell = th.data() + 2 * L * d + 2 * L;
        h.w0 = th[2 * L * d + 2 * L + d];
    }
    if (h0.family == GP2S_KERNEL_FARFIELD) {
        h.ell = th.data() + L * d + 2 * L;
        h.w0 = th[L * d + 2 * L + 1];
    }
    h.r = th[P - 2];
    h.sigma2 = th[P - 1];
    return h;
}

std::vector<double> theta_of(const gp2s_hyper &h0)
{
    const int L = h0.L, d = h0.d;
    std::vector<double> th;
    for (int k = 0; k < L * d; ++k) th.push_back(h0.centers[k]);
    for (int l = 0; l < L; ++l) th.push_back(h0.radii[l]);
    for (int l = 0; l < L; ++l) th.push_back(h0.amps[l]);
    if (h0.family == GP2S_KERNEL_WENDCONV) {
        for (int k = 0; k < L * d; ++k) th.push_back(h0.G[k]);
        for (int k = 0; k < d; ++k) th.push_back(h0.ell[k]);
        th.push_back(h0.w0);
    }
    if (h0.family == GP2S_KERNEL_FARFIELD) {
        th.push_back(h0.ell[0]);
        th.push_back(h0.w0);
    }
    th.push_back(h0.r);
    th.push_back(h0.sigma2);
    return th;
}

bool write_checkpoint(const char *path, int done, const std::vector<double> &th, double lml,
                      const std::vector<int> &acc_blocks)
{
    const std::string tmp = std::string(path) + ".tmp";
    FILE *f = std::fopen(tmp.c_str(), "w");
    if (!f) return false;
    std::fprintf(f, "gp2s-mcmc 1\n%d %d %d\n%.17g\n", done, (int)th.size(), (int)acc_blocks.size(), lml);
    for (size_t p = 0; p < th.size(); ++p) std::fprintf(f, "%.17g%c", th[p], p + 1 == th.size() ? '\n' : ' ');
    for (size_t b = 0; b < acc_blocks.size(); ++b)
        std::fprintf(f, "%d%c", acc_blocks[b], b + 1 == acc_blocks.size() ? '\n' : ' ');
    const bool ok = std::fflush(f) == 0;
    std::fclose(f);
    return ok && std::rename(tmp.c_str(), path) == 0;
}

bool read_checkpoint(const char *path, int P, int nb, int *done, std::vector<double> &th, double *lml,
                     std::vector<int> &acc_blocks)
{
    FILE *f = std::fopen(path, "r");
    if (!f) return false;
    char magic[32] = {0};
    int ver = 0, p_ = 0, nb_ = 0;
    bool ok = std::fscanf(f, "%31s %d", magic, &ver) == 2 && std::strcmp(magic, "gp2s-mcmc") == 0 && ver == 1 &&
              std::fscanf(f, "%d %d %d", done, &p_, &nb_) == 3 && p_ == P && nb_ == nb &&
              std::fscanf(f, "%lf", lml) == 1;
    for (int p = 0; ok && p < P; ++p) ok = std::fscanf(f, "%lf", &th[p]) == 1;
    for (int b = 0; ok && b < nb; ++b) ok = std::fscanf(f, "%d", &acc_blocks[b]) == 1;
    std::fclose(f);
    return ok;
}

}  // namespace

gp2s_status mcmc_run(gp2s_ctx *c, int64_t n, const double *X, const double *y, const gp2s_hyper *h0,
                     const gp2s_opts *o, const gp2s_mcmc_opts *mo, double *chain, int32_t *accept,
                     gp2s_mcmc_info *info)
{
    if (!h0 || !mo || !chain) return set_err(c, GP2S_EINVAL, "hyper / mcmc options / chain is NULL");
    const int L = h0->L, d = h0->d;
    if (d < 1 || d > kMaxDim || L < 0 || L > kMaxBumps) return set_err(c, GP2S_EINVAL, "bad d / L");
    const int P = gp2s_num_params_family(d, L, h0->family);
    const int nb = mo->nblocks;
    if (mo->iters < 0 || nb < 1 || nb > 64 || !mo->block || !mo->step)
        return set_err(c, GP2S_EINVAL, "iters >= 0, 1 <= nblocks <= 64, block and step arrays required");
    for (int p = 0; p < P; ++p) {
        if (mo->block[p] < -1 || mo->block[p] >= nb) return set_err(c, GP2S_EINVAL, "block ids must be in -1..nblocks-1");
        if (!(mo->step[p] >= 0.0) || !std::isfinite(mo->step[p])) return set_err(c, GP2S_EINVAL, "steps must be finite and >= 0");
    }
    if (mo->checkpoint_every < 0) return set_err(c, GP2S_EINVAL, "checkpoint_every must be >= 0");
    gp2s_opts opts = *o;
    opts.pattern_cache = 0;
    std::vector<double> th = theta_of(*h0);
    std::vector<int> acc_blocks(nb, 0);
    int start = 0;
    double cur = 0.0;
    int evals = 0, reused = 0;
    if (mo->resume) {
        if (!mo->checkpoint) return set_err(c, GP2S_EINVAL, "resume needs a checkpoint path");
        if (!read_checkpoint(mo->checkpoint, P, nb, &start, th, &cur, acc_blocks))
            return set_err(c, GP2S_EINVAL, std::string("cannot read checkpoint ") + mo->checkpoint);
        if (start > mo->iters) return set_err(c, GP2S_EINVAL, "checkpoint is past iters");
    } else {
        gp2s_hyper h = hyper_from(*h0, th);
        gp2s_lml_info li;
        GP2S_TRY(lml_single(c, n, X, y, &h, &opts, &cur, nullptr, &li));
        ++evals;
        reused += li.pattern_reused;
    }
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    cudaEventRecord(e0, c->stream);
    std::vector<double> prop(P);
    for (int t = start; t < mo->iters; ++t) {
        for (int b = 0; b < nb; ++b) {
            bool moved = false, inside = true;
            for (int p = 0; p < P; ++p) {
                prop[p] = th[p];
                if (mo->block[p] != b) continue;
                const double z = mo->normals ? mo->normals[(int64_t)t * P + p] : std_normal(mo->seed, (uint64_t)t * P + p);
                prop[p] = th[p] + mo->step[p] * z;
                moved = true;
                if ((mo->lower && prop[p] < mo->lower[p]) || (mo->upper && prop[p] > mo->upper[p])) inside = false;
            }
            int acc = 0;
            if (moved && inside) {
                gp2s_hyper h = hyper_from(*h0, prop);
                double val = 0.0;
                gp2s_lml_info li;
                gp2s_status st = lml_single(c, n, X, y, &h, &opts, &val, nullptr, &li);
                if (st != GP2S_OK && st != GP2S_ENOTPD && st != GP2S_EINVAL) return st;
                ++evals;
                if (st == GP2S_OK) {
                    reused += li.pattern_reused;
                    const double u = mo->uniforms ? mo->uniforms[(int64_t)t * nb + b]
                                                  : unit_uniform(mo->seed, 2, (uint64_t)t * nb + b);
                    const double logu = u > 0.0 ? std::log(u) : -INFINITY;
                    if (logu < val - cur) {
                        th = prop;
                        cur = val;
                        acc = 1;
                        ++acc_blocks[b];
                    }
                }
                // a proposal the engine rejects as invalid (a non-positive-definite A, a
                // non-positive radius) has zero prior density: it is a rejection
            }
            if (accept) accept[(int64_t)t * nb + b] = acc;
        }
        for (int p = 0; p < P; ++p) chain[(int64_t)t * (P + 1) + p] = th[p];
        chain[(int64_t)t * (P + 1) + P] = cur;
        const bool ckpt = mo->checkpoint && mo->checkpoint_every > 0 &&
                          ((t + 1) % mo->checkpoint_every == 0 || t + 1 == mo->iters);
        if (ckpt && !write_checkpoint(mo->checkpoint, t + 1, th, cur, acc_blocks))
            return set_err(c, GP2S_EINVAL, std::string("cannot write checkpoint ") + mo->checkpoint + ": " +
                                               std::strerror(errno));
    }
    cudaEventRecord(e1, c->stream);
    cudaEventSynchronize(e1);
    if (info) {
        std::memset(info, 0, sizeof(*info));
        info->start = start;
        info->done = mo->iters;
        info->evals = evals;
        info->pattern_reused = reused;
        int tot = 0;
        for (int b = 0; b < nb; ++b) tot += acc_blocks[b];
        info->accepted = tot;
        info->lml = cur;
        cudaEventElapsedTime(&info->ms, e0, e1);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    c->err.clear();
    return GP2S_OK;
}

}  // namespace gp2s
