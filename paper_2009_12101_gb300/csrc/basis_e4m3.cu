// basis_e4m3.cu -- kernels of the E4M3 basis format (explicit instantiation).
#include "cbg_launch_impl.cuh"
namespace cbg {
template struct Launcher<E4M3>;
}  // namespace cbg
