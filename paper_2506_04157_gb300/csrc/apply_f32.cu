// F32 instantiations of the fused micro-tet sweep.
#include "apply_launch.cuh"

namespace mfs {
template mfs_status launch_apply<float>(mfs_problem*, int, int, int, int, const float*, const float*, float*, float*,
                                       const float*, int, int, int);
template ApplyParams<float> fill_params<float>(mfs_problem*, int, int, const float*, const float*, float*, float*,
                                                const float*);
template mfs_status launch_batch<float>(const ApplyParams<float>*, const int2*, const int*, int, int, int, cudaStream_t);
}  // namespace mfs
