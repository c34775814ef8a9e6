// basis_i16.cu -- kernels of the I16 basis format (explicit instantiation).
#include "cbg_launch_impl.cuh"
namespace cbg {
template struct Launcher<I16>;
}  // namespace cbg
