// basis_f32.cu -- kernels of the F32 basis format (explicit instantiation).
#include "cbg_launch_impl.cuh"
namespace cbg {
template struct Launcher<F32>;
}  // namespace cbg
