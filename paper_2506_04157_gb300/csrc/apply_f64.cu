// F64 instantiations of the fused micro-tet sweep.
#include "apply_launch.cuh"

namespace mfs {
template mfs_status launch_apply<double>(mfs_problem*, int, int, int, int, const double*, const double*, double*, double*,
                                       const double*, int, int, int);
template ApplyParams<double> fill_params<double>(mfs_problem*, int, int, const double*, const double*, double*, double*,
                                                const double*);
template mfs_status launch_batch<double>(const ApplyParams<double>*, const int2*, const int*, int, int, int, cudaStream_t);
}  // namespace mfs
