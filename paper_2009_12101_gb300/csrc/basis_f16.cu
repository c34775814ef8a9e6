// basis_f16.cu -- kernels of the F16 basis format (explicit instantiation).
#include "cbg_launch_impl.cuh"
namespace cbg {
template struct Launcher<F16>;
}  // namespace cbg
