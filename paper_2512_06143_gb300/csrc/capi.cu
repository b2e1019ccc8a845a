// capi.cu -- the extern "C" entry points of include/gp2s.h: context and workspace management,
// host/device input staging, and the orchestration of assemble -> solve -> log-det -> LML
// (Sec. 3) -> adjoint gradient.
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <utility>

#include "gp2s_internal.cuh"

namespace gp2s {

gp2s_status validate_hyper(gp2s_ctx *c, const gp2s_hyper *h);   // assemble.cu
gp2s_status y_residual(gp2s_ctx *c, const double *y_sorted_dev, double *relres);   // krylov.cu

gp2s_status set_err(gp2s_ctx *c, gp2s_status st, const std::string &msg)
{
    if (c) c->err = msg;
    return st;
}

gp2s_status cuda_err(gp2s_ctx *c, cudaError_t e, const char *where)
{
    std::string m = std::string("CUDA error ") + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ") at " + where;
    if (e == cudaErrorMemoryAllocation) return set_err(c, GP2S_ENOMEM, m);
    return set_err(c, GP2S_ECUDA, m);
}

gp2s_status ensure(gp2s_ctx *c, DevBuf &b, size_t bytes)
{
    if (bytes == 0) bytes = 16;
    if (b.bytes >= bytes) return GP2S_OK;
    if (c->mem_limit && c->mem_in_use - b.bytes + bytes > c->mem_limit)
        return set_err(c, GP2S_ENOMEM, "GP2S_MEM_LIMIT exceeded");
    if (b.p) {
        cudaError_t e = cudaFree(b.p);
        if (e != cudaSuccess) return cuda_err(c, e, "cudaFree");
        c->mem_in_use -= b.bytes;
        b.p = nullptr;
        b.bytes = 0;
    }
    size_t alloc = (bytes + 255) & ~size_t(255);
    cudaError_t e = cudaMalloc(&b.p, alloc);
    if (e != cudaSuccess) {
        b.p = nullptr;
        cudaGetLastError();
        return cuda_err(c, e, "cudaMalloc");
    }
    b.bytes = alloc;
    c->mem_in_use += alloc;
    return GP2S_OK;
}

gp2s_status smem_attr(gp2s_ctx *c, const void *func, size_t smem)
{
    // The attribute belongs to the function on this device, shared by every context and host
    // thread (the batched engine runs several at once): it only ever grows, under a lock, so a
    // launch sized for an earlier, larger request is never invalidated by a smaller one.
    static std::mutex mu;
    static std::map<std::pair<int, const void *>, size_t> set;
    std::lock_guard<std::mutex> lk(mu);
    size_t &cur = set[std::make_pair(c->device, func)];
    if (smem <= cur) return GP2S_OK;
    GP2S_CUDA(c, cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    cur = smem;
    return GP2S_OK;
}

gp2s_status ensure_host(gp2s_ctx *c, HostPinned &b, size_t bytes)
{
    if (b.bytes >= bytes) return GP2S_OK;
    if (b.p) cudaFreeHost(b.p);
    b.p = nullptr;
    b.bytes = 0;
    cudaError_t e = cudaMallocHost(&b.p, bytes);
    if (e != cudaSuccess) return cuda_err(c, e, "cudaMallocHost");
    b.bytes = bytes;
    return GP2S_OK;
}

static void free_buf(DevBuf &b)
{
    if (b.p) cudaFree(b.p);
    b.p = nullptr;
    b.bytes = 0;
}

static bool is_device_ptr(const void *p)
{
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// Make `src` (host or device, `bytes` long) available on the device; returns the device pointer.
static gp2s_status stage_in(gp2s_ctx *c, DevBuf &buf, const void *src, size_t bytes, const void **dev)
{
    if (is_device_ptr(src)) {
        *dev = src;
        return GP2S_OK;
    }
    GP2S_TRY(ensure(c, buf, bytes));
    GP2S_CUDA(c, cudaMemcpyAsync(buf.p, src, bytes, cudaMemcpyHostToDevice, c->stream));
    *dev = buf.p;
    return GP2S_OK;
}

__global__ void k_gather_sorted(int64_t n, const int32_t *__restrict__ perm, const double *__restrict__ src,
                                double *__restrict__ dst)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        dst[i] = src[perm[i]];
}

__global__ void k_scatter_orig(int64_t n, const int32_t *__restrict__ perm, const double *__restrict__ src,
                               double *__restrict__ dst)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        dst[perm[i]] = src[i];
}

__global__ void k_check_finite(int64_t n, const double *__restrict__ v, int *__restrict__ bad)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        if (!isfinite(v[i])) atomicOr(bad, 1);
}

// y (original order, host or device) -> c->ys64 (sorted order, device).  Checks finiteness.
static gp2s_status stage_y(gp2s_ctx *c, const double *y)
{
    const int64_t n = c->A.n;
    const void *yd = nullptr;
    GP2S_TRY(stage_in(c, c->yin, y, sizeof(double) * n, &yd));
    GP2S_TRY(ensure(c, c->ys64, sizeof(double) * n));
    GP2S_TRY(ensure(c, c->counters, 256));
    int *bad = reinterpret_cast<int *>(c->counters.as<char>() + 200);
    GP2S_CUDA(c, cudaMemsetAsync(bad, 0, sizeof(int), c->stream));
    unsigned gb = (unsigned)std::min<int64_t>(ceil_div(n, 256), 152 * 8);
    k_check_finite<<<gb, 256, 0, c->stream>>>(n, (const double *)yd, bad);
    GP2S_LAUNCH(c);
    k_gather_sorted<<<gb, 256, 0, c->stream>>>(n, c->perm.as<int32_t>(), (const double *)yd, c->ys64.as<double>());
    GP2S_LAUNCH(c);
    int hb = 0;
    GP2S_CUDA(c, cudaMemcpyAsync(&hb, bad, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    GP2S_CUDA(c, cudaStreamSynchronize(c->stream));
    if (hb) return set_err(c, GP2S_EINVAL, "y contains NaN or infinity");
    return GP2S_OK;
}

static gp2s_status validate_opts(gp2s_ctx *c, const gp2s_opts *o)
{
    if (!o) return set_err(c, GP2S_EINVAL, "opts is NULL");
    if (o->precision != GP2S_PREC_FP64 && o->precision != GP2S_PREC_MIXED) return set_err(c, GP2S_EINVAL, "bad precision");
    if (o->logdet < GP2S_LOGDET_AUTO || o->logdet > GP2S_LOGDET_SLQ) return set_err(c, GP2S_EINVAL, "bad logdet method");
    if (!(o->probes == 0 || o->probes == 16 || o->probes == 32 || o->probes == 48 || o->probes == 64 ||
          o->probes == 96 || o->probes == 128))
        return set_err(c, GP2S_EINVAL, "probes must be 0, 16, 32, 48, 64, 96 or 128");
    if (o->lanczos_steps < 1 || o->lanczos_steps > 4096) return set_err(c, GP2S_EINVAL, "lanczos_steps must be in 1..4096");
    if (o->max_iter < 1) return set_err(c, GP2S_EINVAL, "max_iter must be >= 1");
    if (!(o->tol_inner > 0.0) || !(o->tol_refine > 0.0) || !(o->tol_probe > 0.0)) return set_err(c, GP2S_EINVAL, "tolerances must be > 0");
    if (o->max_outer < 0) return set_err(c, GP2S_EINVAL, "max_outer must be >= 0");
    if (o->precond < 0 || o->precond > 2) return set_err(c, GP2S_EINVAL, "precond must be 0, 1 or 2");
    if (o->solver != GP2S_SOLVER_CG && o->solver != GP2S_SOLVER_MINRES) return set_err(c, GP2S_EINVAL, "unknown solver");
    if (o->bj_block != 0 && o->bj_block != 64 && o->bj_block != 128)
        return set_err(c, GP2S_EINVAL, "bj_block must be 0, 64 or 128");
    return GP2S_OK;
}

static int logdet_method(const gp2s_opts *o, int64_t n)
{
    if (o->logdet == GP2S_LOGDET_AUTO) return n <= o->n_exact ? GP2S_LOGDET_EXACT : GP2S_LOGDET_SLQ;
    return o->logdet;
}

struct Ev {
    cudaEvent_t e = nullptr;
    Ev() { cudaEventCreate(&e); }
    ~Ev() { if (e) cudaEventDestroy(e); }
};

static float elapsed(cudaEvent_t a, cudaEvent_t b)
{
    float ms = 0.0f;
    cudaEventElapsedTime(&ms, a, b);
    return ms;
}

static gp2s_status do_assemble(gp2s_ctx *c, int64_t n, const double *X, const gp2s_hyper *h, const gp2s_opts *o)
{
    if (n < 1) return set_err(c, GP2S_EINVAL, "n must be >= 1");
    if (n > (int64_t)INT32_MAX - 1) return set_err(c, GP2S_EOVERFLOW, "n exceeds the int32 index range");
    if (!X) return set_err(c, GP2S_EINVAL, "X is NULL");
    GP2S_TRY(validate_hyper(c, h));
    GP2S_TRY(validate_opts(c, o));
    const void *xd = nullptr;
    GP2S_TRY(stage_in(c, c->Xin, X, sizeof(double) * (size_t)n * h->d, &xd));
    return assemble_problem(c, n, (const double *)xd, h, o);
}

// Solve (and probe CG when m > 0) on the assembled problem with y already in c->ys64.
static gp2s_status do_solve(gp2s_ctx *c, int method, int m, CGResult *res)
{
    const Assembled &A = c->A;
    if (method == GP2S_LOGDET_EXACT && m == 0 && A.opts.solver == GP2S_SOLVER_CG) {
        double ld = 0.0;
        GP2S_TRY(exact_logdet_solve(c, c->ys64.as<double>(), &ld, false));
        double rr = 0.0;
        GP2S_TRY(y_residual(c, c->ys64.as<double>(), &rr));
        res->relres = rr;
        res->iters_y = 0;
        res->outer = 0;
        c->solve_relres = rr;
        c->have_solution = true;
        return GP2S_OK;
    }
    return krylov_solve(c, c->ys64.as<double>(), m > 0, m, A.opts.lanczos_steps, res);
}

}  // namespace gp2s

using namespace gp2s;

extern "C" {

void gp2s_opts_default(gp2s_opts *o)
{
    if (!o) return;
    std::memset(o, 0, sizeof(*o));
    o->precision = GP2S_PREC_MIXED;
    o->logdet = GP2S_LOGDET_AUTO;
    o->n_exact = 20000;
    o->probes = 64;
    o->lanczos_steps = 100;
    o->max_iter = 20000;
    o->tol_inner = 1e-6;
    o->tol_refine = 1e-8;
    o->tol_probe = 1e-5;
    o->seed = 0;
    o->precond = 2;
    o->exact_support = 0;
    o->max_outer = 8;
}

int32_t gp2s_num_params(int32_t d, int32_t L) { return L * (d + 2) + 2; }

int32_t gp2s_num_params_family(int32_t d, int32_t L, int32_t family)
{
    if (family == GP2S_KERNEL_WENDCONV) return L * (2 * d + 2) + d + 3;
    if (family == GP2S_KERNEL_FARFIELD) return L * (d + 2) + 4;
    return L * (d + 2) + 2;
}

gp2s_status gp2s_create(gp2s_ctx **ctx, int device, void *cuda_stream)
{
    if (!ctx) return GP2S_EINVAL;
    *ctx = nullptr;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
        cudaGetLastError();
        return GP2S_ECUDA;
    }
    if (cudaSetDevice(device) != cudaSuccess) return GP2S_ECUDA;
    gp2s_ctx *c = new gp2s_ctx();
    c->device = device;
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) == cudaSuccess && sms > 0) c->num_sms = sms;
    c->stream = reinterpret_cast<cudaStream_t>(cuda_stream);
    const char *bw = std::getenv("GP2S_BATCH_WORKERS");
    if (bw && std::atoi(bw) > 0) c->batch_workers_max = std::atoi(bw);
    const char *lim = std::getenv("GP2S_MEM_LIMIT");
    if (lim) c->mem_limit = (size_t)std::strtoull(lim, nullptr, 10);
    const char *gr = std::getenv("GP2S_GRAPHS");
    if (gr && std::strcmp(gr, "0") == 0) c->use_graphs = false;
    const char *pa = std::getenv("GP2S_PC_ASYNC");
    if (pa && std::strcmp(pa, "0") == 0) c->pc_async = false;
    const char *ry = std::getenv("GP2S_RELIABLE_Y");
    if (ry && std::strcmp(ry, "0") == 0) c->reliable_y = false;
    const char *p64 = std::getenv("GP2S_PC_ASYNC64");
    if (p64 && std::strcmp(p64, "0") == 0) c->pc_async64 = false;
    const char *sa = std::getenv("GP2S_SLQ_ASYNC");
    if (sa && std::strcmp(sa, "0") == 0) c->slq_async = false;
    const char *rm = std::getenv("GP2S_RELIABLE_MIN_ROWS");
    if (rm && std::atoll(rm) >= 0) c->reliable_min_rows = (int64_t)std::atoll(rm);
    const char *rd = std::getenv("GP2S_RELIABLE_DELTA");
    if (rd && std::atof(rd) > 0.0 && std::atof(rd) < 1.0) c->reliable_delta = std::atof(rd);
    const char *fy = std::getenv("GP2S_PC_FUSE_Y");
    if (fy && std::strcmp(fy, "0") == 0) c->pc_fuse_y = false;
    const char *sh = std::getenv("GP2S_SPMM_HALF");
    if (sh && std::strcmp(sh, "1") == 0) c->spmm_half = true;
    const char *st = std::getenv("GP2S_SPMM_TMA");
    if (st) c->spmm_tma = std::atoi(st);
    *ctx = c;
    return GP2S_OK;
}

void gp2s_destroy(gp2s_ctx *c)
{
    if (!c) return;
    cudaSetDevice(c->device);
    if (c->stream) cudaStreamSynchronize(c->stream);
    DevBuf *bufs[] = {&c->Xin, &c->yin, &c->keys, &c->keys2, &c->idx, &c->idx2, &c->perm, &c->iperm,
                      &c->Xs64, &c->Xhi, &c->Xlo, &c->ys64, &c->bbox_part, &c->bbox, &c->hist,
                      &c->scan_tmp, &c->scan_tmp2, &c->cell_start, &c->cell_flag, &c->items, &c->item_cnt,
                      &c->B64, &c->B32, &c->D64, &c->s64, &c->s32, &c->rowcnt, &c->rowptr, &c->col,
                      &c->val32, &c->val64, &c->counters, &c->vec, &c->vec64, &c->partials, &c->scal,
                      &c->Z, &c->Zf, &c->rec, &c->rsplit, &c->dense, &c->H, &c->gpart,
                      &c->rb_cnt, &c->rb_ptr, &c->rb_col, &c->rb_val, &c->rb_tpart, &c->rb_seg,
                      &c->bj_Minv, &c->bj_ld, &c->bj_Minv_y, &c->post_X, &c->post_B, &c->post_cnt,
                      &c->post_part, &c->mr_vec, &c->mc_X, &c->mc_y, &c->wc_lam, &c->wc_sig, &c->ff_mask,
                      &c->ff_flag, &c->ff_mptr, &c->ff_mcol, &c->ff_ucnt, &c->ff_uptr, &c->ff_ucol};
    for (DevBuf *b : bufs) free_buf(*b);
    for (cudaEvent_t e : c->prof_ev) cudaEventDestroy(e);
    for (gp2s_ctx *w : c->workers) gp2s_destroy(w);
    for (cudaStream_t s : c->worker_streams) cudaStreamDestroy(s);
    if (c->capture_stream) cudaStreamDestroy(c->capture_stream);
    if (c->side_stream) {
        cudaStreamSynchronize(c->side_stream);
        cudaStreamDestroy(c->side_stream);
    }
    if (c->slq_ev_rec) cudaEventDestroy(c->slq_ev_rec);
    if (c->slq_ev_done) cudaEventDestroy(c->slq_ev_done);
    free_buf(c->slq_work);
    if (c->hbuf.p) cudaFreeHost(c->hbuf.p);
    delete c;
}

const char *gp2s_last_error(const gp2s_ctx *c) { return c ? c->err.c_str() : "null context"; }

gp2s_status gp2s_assemble(gp2s_ctx *c, int64_t n, const double *X, const gp2s_hyper *h, const gp2s_opts *o,
                          gp2s_assemble_info *info)
{
    if (!c) return GP2S_EINVAL;
    c->err.clear();
    if (cudaSetDevice(c->device) != cudaSuccess) return cuda_err(c, cudaGetLastError(), "cudaSetDevice");
    gp2s_opts def;
    if (!o) { gp2s_opts_default(&def); o = &def; }
    GP2S_TRY(do_assemble(c, n, X, h, o));
    if (info) *info = c->A.info;
    return GP2S_OK;
}

gp2s_status gp2s_csr(gp2s_ctx *c, gp2s_csr_view *v)
{
    if (!c || !v) return GP2S_EINVAL;
    if (!c->A.valid) return set_err(c, GP2S_ENOTREADY, "nothing assembled");
    v->n = c->A.n;
    v->nnz = c->A.nnz;
    v->rowptr = c->rowptr.as<int32_t>();
    v->col = c->col.as<int32_t>();
    v->perm = c->perm.as<int32_t>();
    v->val32 = c->A.precision == GP2S_PREC_MIXED ? c->val32.as<float>() : nullptr;
    v->val64 = c->val64.as<double>();
    v->dscale = c->s64.as<double>();
    return GP2S_OK;
}

gp2s_status gp2s_solve(gp2s_ctx *c, const double *y, double *a, gp2s_solve_info *info)
{
    if (!c) return GP2S_EINVAL;
    c->err.clear();
    if (!c->A.valid) return set_err(c, GP2S_ENOTREADY, "gp2s_solve needs gp2s_assemble first");
    if (!y || !a) return set_err(c, GP2S_EINVAL, "y / a is NULL");
    if (cudaSetDevice(c->device) != cudaSuccess) return cuda_err(c, cudaGetLastError(), "cudaSetDevice");
    Ev e0, e1;
    cudaEventRecord(e0.e, c->stream);
    GP2S_TRY(stage_y(c, y));
    CGResult res;
    gp2s_status st = krylov_solve(c, c->ys64.as<double>(), false, 0, 1, &res);
    if (st != GP2S_OK && st != GP2S_ENOCONV) return st;
    const int64_t n = c->A.n;
    // a (original order) <- a_sorted
    const double *as = c->vec64.as<double>() + 3 * n;
    unsigned gb = (unsigned)std::min<int64_t>(ceil_div(n, 256), 152 * 8);
    if (is_device_ptr(a)) {
        k_scatter_orig<<<gb, 256, 0, c->stream>>>(n, c->perm.as<int32_t>(), as, a);
        GP2S_LAUNCH(c);
    } else {
        GP2S_TRY(ensure(c, c->yin, sizeof(double) * n));
        k_scatter_orig<<<gb, 256, 0, c->stream>>>(n, c->perm.as<int32_t>(), as, c->yin.as<double>());
        GP2S_LAUNCH(c);
        GP2S_CUDA(c, cudaMemcpyAsync(a, c->yin.p, sizeof(double) * n, cudaMemcpyDeviceToHost, c->stream));
    }
    cudaEventRecord(e1.e, c->stream);
    GP2S_CUDA(c, cudaStreamSynchronize(c->stream));
    if (info) {
        info->iters = res.iters_y;
        info->outer = res.outer;
        info->relres = res.relres;
        info->ms = elapsed(e0.e, e1.e);
    }
    return st;
}

gp2s_status gp2s_logdet(gp2s_ctx *c, double *logdet, double *stderr_hat, gp2s_logdet_info *info)
{
    if (!c) return GP2S_EINVAL;
    c->err.clear();
    if (!c->A.valid) return set_err(c, GP2S_ENOTREADY, "gp2s_logdet needs gp2s_assemble first");
    if (!logdet) return set_err(c, GP2S_EINVAL, "logdet is NULL");
    if (cudaSetDevice(c->device) != cudaSuccess) return cuda_err(c, cudaGetLastError(), "cudaSetDevice");
    const Assembled &A = c->A;
    const int method = logdet_method(&A.opts, A.n);
    Ev e0, e1;
    cudaEventRecord(e0.e, c->stream);
    double ldiag = 0.0, lhat = 0.0, se = 0.0;
    GP2S_TRY(sum_log_diag(c, &ldiag));
    if (method == GP2S_LOGDET_EXACT) {
        GP2S_TRY(exact_logdet_solve(c, nullptr, &lhat, false));
    } else {
        const int m = A.opts.probes;
        if (m <= 0) return set_err(c, GP2S_EINVAL, "SLQ needs probes > 0");
        GP2S_TRY(ensure(c, c->ys64, sizeof(double) * A.n));
        GP2S_CUDA(c, cudaMemsetAsync(c->ys64.p, 0, sizeof(double) * A.n, c->stream));
        CGResult res;
        gp2s_status st = krylov_solve(c, c->ys64.as<double>(), true, m, A.opts.lanczos_steps, &res);
        if (st != GP2S_OK && st != GP2S_ENOCONV) return st;
        c->have_solution = false;
        GP2S_TRY(slq_logdet(c, m, A.opts.lanczos_steps, &lhat, &se));
    }
    cudaEventRecord(e1.e, c->stream);
    GP2S_CUDA(c, cudaStreamSynchronize(c->stream));
    *logdet = ldiag + lhat;
    if (stderr_hat) *stderr_hat = se;
    if (info) {
        info->method = method;
        info->probes = method == GP2S_LOGDET_SLQ ? A.opts.probes : 0;
        info->steps = method == GP2S_LOGDET_SLQ ? A.opts.lanczos_steps : 0;
        info->logdet_diag = ldiag;
        info->logdet_hat = lhat;
        info->stderr_hat = se;
        info->ms = elapsed(e0.e, e1.e);
    }
    return GP2S_OK;
}

static gp2s_status lml_impl(gp2s_ctx *c, int64_t n, const double *X, const double *y, const gp2s_hyper *h,
                            const gp2s_opts *o, double *lml, double *grad, gp2s_lml_info *info)
{
    if (!c) return GP2S_EINVAL;
    c->err.clear();
    if (!lml) return set_err(c, GP2S_EINVAL, "lml is NULL");
    if (!y) return set_err(c, GP2S_EINVAL, "y is NULL");
    if (cudaSetDevice(c->device) != cudaSuccess) return cuda_err(c, cudaGetLastError(), "cudaSetDevice");
    gp2s_opts def;
    if (!o) { gp2s_opts_default(&def); o = &def; }
    c->launches = 0;
    c->spmm_launches = 0;
    c->spmm_bytes = 0.0;
    c->spmm_seg_tiles = 0;
    c->prof_ms = 0.0;
    c->prof_used = 0;
    c->profile = o->profile != 0;
    Ev e0, e1, e2, e3, e4;
    cudaEventRecord(e0.e, c->stream);
    GP2S_TRY(do_assemble(c, n, X, h, o));
    cudaEventRecord(e1.e, c->stream);
    const Assembled &A = c->A;
    const int method = logdet_method(o, n);
    const int m = (grad || method == GP2S_LOGDET_SLQ) ? o->probes : 0;
    if ((grad || method == GP2S_LOGDET_SLQ) && m <= 0) return set_err(c, GP2S_EINVAL, "SLQ / gradient need probes > 0");
    GP2S_TRY(stage_y(c, y));
    CGResult res;
    c->probes_for_grad = grad != nullptr;
    gp2s_status st = do_solve(c, method, m, &res);
    c->probes_for_grad = false;
    if (st != GP2S_OK) return st;
    cudaEventRecord(e2.e, c->stream);
    double ldiag = 0.0, lhat = 0.0, se = 0.0;
    GP2S_TRY(sum_log_diag(c, &ldiag));
    if (method == GP2S_LOGDET_EXACT) {
        if (c->have_exact) lhat = c->exact_lhat;      // factored by the dense solve
        else GP2S_TRY(exact_logdet_solve(c, nullptr, &lhat, false));
    } else {
        GP2S_TRY(slq_logdet(c, m, o->lanczos_steps, &lhat, &se));
    }
    cudaEventRecord(e3.e, c->stream);
    double quad = 0.0;
    GP2S_TRY(dot_f64(c, c->ys64.as<double>(), c->vec64.as<double>() + 3 * A.n, A.n, &quad));
    const double logdet = ldiag + lhat;
    const double val = -0.5 * quad - 0.5 * logdet - 0.5 * (double)A.n * std::log(2.0 * M_PI);
    if (grad) GP2S_TRY(adjoint_gradient(c, m, grad));
    cudaEventRecord(e4.e, c->stream);
    GP2S_CUDA(c, cudaStreamSynchronize(c->stream));
    *lml = val;
    if (info) {
        std::memset(info, 0, sizeof(*info));
        info->lml = val;
        info->quad = quad;
        info->logdet = logdet;
        info->logdet_stderr = se;
        info->relres = res.relres;
        info->n = A.n;
        info->nnz = A.nnz;
        info->iters_y = res.iters_y;
        info->iters_probes = res.iters_probes;
        info->outer = res.outer;
        info->logdet_method = method;
        info->ms_assemble = elapsed(e0.e, e1.e);
        info->ms_solve = elapsed(e1.e, e2.e);
        info->ms_logdet = elapsed(e2.e, e3.e);
        info->ms_grad = elapsed(e3.e, e4.e);
        info->ms_total = elapsed(e0.e, e4.e);
        info->launches = c->launches;
        info->spmm_launches = c->spmm_launches;
        info->spmm_bytes = c->spmm_bytes;
        info->ms_spmm = (float)c->prof_ms;
        info->bj_block = (A.precision == GP2S_PREC_MIXED && A.opts.precond == 2 && c->bj_valid) ? c->bj_size : 0;
        info->spmm_seg_tiles = c->spmm_seg_tiles;
        info->pattern_reused = A.info.pattern_reused;
        info->batch_config = -1;
    }
    c->profile = false;
    return GP2S_OK;
}

gp2s_status gp2s_lml(gp2s_ctx *c, int64_t n, const double *X, const double *y, const gp2s_hyper *h,
                     const gp2s_opts *o, double *lml, gp2s_lml_info *info)
{
    return lml_impl(c, n, X, y, h, o, lml, nullptr, info);
}

gp2s_status gp2s_lml_batched(gp2s_ctx *c, int32_t B, const int64_t *n, const double *const *X,
                             const double *const *y, const gp2s_hyper *hyper, const gp2s_opts *opts,
                             double *lml_host, gp2s_lml_info *info_host)
{
    return batched_lml(c, B, n, X, y, hyper, opts, lml_host, info_host);
}

gp2s_status gp2s_mcmc(gp2s_ctx *c, int64_t n, const double *X, const double *y, const gp2s_hyper *h0,
                      const gp2s_opts *o, const gp2s_mcmc_opts *mo, double *chain, int32_t *accept,
                      gp2s_mcmc_info *info)
{
    if (!c) return GP2S_EINVAL;
    c->err.clear();
    if (cudaSetDevice(c->device) != cudaSuccess) return cuda_err(c, cudaGetLastError(), "cudaSetDevice");
    gp2s_opts def;
    if (!o) { gp2s_opts_default(&def); o = &def; }
    GP2S_TRY(validate_hyper(c, h0));
    GP2S_TRY(validate_opts(c, o));
    if (!X || !y) return set_err(c, GP2S_EINVAL, "X / y is NULL");
    // host inputs are staged once for the whole chain
    const void *xd = nullptr, *yd = nullptr;
    GP2S_TRY(stage_in(c, c->mc_X, X, sizeof(double) * (size_t)n * h0->d, &xd));
    GP2S_TRY(stage_in(c, c->mc_y, y, sizeof(double) * (size_t)n, &yd));
    return mcmc_run(c, n, (const double *)xd, (const double *)yd, h0, o, mo, chain, accept, info);
}

gp2s_status gp2s_posterior(gp2s_ctx *c, int64_t n_test, const double *Xtest, double *mean, double *var,
                           gp2s_posterior_info *info)
{
    if (!c) return GP2S_EINVAL;
    c->err.clear();
    if (cudaSetDevice(c->device) != cudaSuccess) return cuda_err(c, cudaGetLastError(), "cudaSetDevice");
    return posterior(c, n_test, Xtest, mean, var, info);
}

gp2s_status gp2s_lml_grad(gp2s_ctx *c, int64_t n, const double *X, const double *y, const gp2s_hyper *h,
                          const gp2s_opts *o, double *lml, double *grad_host, gp2s_lml_info *info)
{
    if (c && !grad_host) return set_err(c, GP2S_EINVAL, "grad_host is NULL");
    return lml_impl(c, n, X, y, h, o, lml, grad_host, info);
}

}  // extern "C"

namespace gp2s {

// One problem on one (worker) context: the engine of gp2s_lml / gp2s_lml_grad.
gp2s_status lml_single(gp2s_ctx *c, int64_t n, const double *X, const double *y, const gp2s_hyper *h,
                       const gp2s_opts *o, double *lml, double *grad, gp2s_lml_info *info)
{
    return lml_impl(c, n, X, y, h, o, lml, grad, info);
}

}  // namespace gp2s
