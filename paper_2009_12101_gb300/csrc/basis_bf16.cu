// basis_bf16.cu -- kernels of the BF16 basis format (explicit instantiation).
#include "cbg_launch_impl.cuh"
namespace cbg {
template struct Launcher<BF16>;
}  // namespace cbg
