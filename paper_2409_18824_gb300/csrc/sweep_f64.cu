// double instantiations of the star-stencil launchers (kernels in star.cuh).
#include "star.cuh"

namespace stn {

template int launch_star<double>(const double*, const double*, double*, const Grid&, const double*, SweepMode,
                             double*, cudaStream_t, i64, i64*);
template int launch_copy_halo<double>(const double*, double*, const Grid&, cudaStream_t);

}  // namespace stn
