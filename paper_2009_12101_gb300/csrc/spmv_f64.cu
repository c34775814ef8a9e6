// spmv_f64.cu -- SpMV kernels with an FP64 input vector: the explicit residual
// r = b - A x of Fig. 1, the second stage of the preconditioned operator (A z after
// z = P v), and the solution update's x += P t.
#include "cbg_launch_impl.cuh"
namespace cbg {
void spmv_f64(int mode, int group, int grid, cudaStream_t s, const SpmvArgs& a)
{
    if (mode == SPMV_RESIDUAL) { CBG_SPMV_GROUPS(-1, SPMV_RESIDUAL) }
    else if (mode == SPMV_ARNOLDI) { CBG_SPMV_GROUPS(-1, SPMV_ARNOLDI) }
    else if (mode == SPMV_ACCUM) { CBG_SPMV_GROUPS(-1, SPMV_ACCUM) }
    else { CBG_SPMV_GROUPS(-1, SPMV_PLAIN) }
}
void spmv_sell_f64(int grid, cudaStream_t s, const SellArgs& a) { k_spmv_sell<-1><<<grid, THREADS, 0, s>>>(a); }
int spmv_occupancy()
{
    int b = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_spmv<-1, 1, SPMV_RESIDUAL>, THREADS, 0);
    return b;
}
}  // namespace cbg
