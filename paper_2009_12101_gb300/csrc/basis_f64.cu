// basis_f64.cu -- kernels of the F64 basis format (explicit instantiation).
#include "cbg_launch_impl.cuh"
namespace cbg {
template struct Launcher<F64>;
}  // namespace cbg
