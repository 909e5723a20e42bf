// pathfind.cu -- batched source-receiver path finding (placeholder until the kernels land).
#include "rp_internal.h"

namespace rph {
int run_find_paths(rp_medium_t, int64_t, const double *, const double *, const double *,
                   const int32_t *, const rp_path_params *, rp_solutions *, rp_stats *,
                   cudaStream_t)
{
    set_error("rp_find_paths: not built yet");
    return RP_ERR_UNSUPPORTED;
}
}  // namespace rph
