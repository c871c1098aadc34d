// F64 instantiations of the fused micro-tet sweep.
#include "apply_launch.cuh"

namespace mfs {
template mfs_status launch_apply<double>(mfs_problem*, int, int, int, int, const double*, const double*, double*, double*,
                                       const double*);
}  // namespace mfs
