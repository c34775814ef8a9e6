// basis_i32.cu -- kernels of the I32 basis format (explicit instantiation).
#include "cbg_launch_impl.cuh"
namespace cbg {
template struct Launcher<I32>;
}  // namespace cbg
