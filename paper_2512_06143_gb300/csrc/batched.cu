// batched.cu -- many independent problems in one call (see gp2s_lml_batched in include/gp2s.h).
#include "gp2s_internal.cuh"

namespace gp2s {

gp2s_status batched_lml(gp2s_ctx *c, int32_t B, const int64_t *n, const double *const *X,
                        const double *const *y, const gp2s_hyper *hyper, const gp2s_opts *opts,
                        double *lml_host, gp2s_lml_info *info_host)
{
    (void)B; (void)n; (void)X; (void)y; (void)hyper; (void)opts; (void)lml_host; (void)info_host;
    return set_err(c, GP2S_EINVAL, "batched form not built");
}

}  // namespace gp2s
