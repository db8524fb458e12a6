// 2D lattice context (placeholder until the 2D kernels land).
#include "lat2d.h"

namespace lat {
struct Ctx2D { int dummy; };
int ctx2d_create(Ctx2D** out, const lat_grid*, DevState*, int, cudaStream_t) { *out = nullptr; return LAT_EINVAL; }
int ctx2d_set_flow(Ctx2D*, const lat_flow*, bool, cudaStream_t) { return LAT_EINVAL; }
int ctx2d_set_noise(Ctx2D*, const double*, long long, long long, cudaStream_t) { return LAT_EINVAL; }
int ctx2d_step(Ctx2D*, void* const*, int, cudaStream_t) { return LAT_EINVAL; }
int ctx2d_prepare(Ctx2D*, void* const*, int) { return LAT_EINVAL; }
int ctx2d_moments(Ctx2D*, const void*, double*, double*, double*, double*, cudaStream_t) { return LAT_EINVAL; }
int ctx2d_set_launch(Ctx2D*, int, int, int, int) { return LAT_EINVAL; }
int ctx2d_autotune(Ctx2D*, void* const*, int, double*, cudaStream_t) { return LAT_EINVAL; }
void ctx2d_destroy(Ctx2D* c) { delete c; }
}  // namespace lat
