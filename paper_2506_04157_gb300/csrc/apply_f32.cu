// F32 instantiations of the fused micro-tet sweep.
#include "apply_launch.cuh"

namespace mfs {
template mfs_status launch_apply<float>(mfs_problem*, int, int, int, int, const float*, const float*, float*, float*,
                                       const float*);
}  // namespace mfs
