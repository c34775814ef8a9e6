// cbg_launch.h -- declarations of the host-side kernel launchers.  The definitions live
// in cbg_launch_impl.cuh and are instantiated once per basis format (basis_<fmt>.cu), so
// the seven formats compile in parallel.
#pragma once
#include <cuda_runtime.h>

#include "cbg_batched.cuh"
#include "cbg_kernels.cuh"
#include "cbg_stream.cuh"

namespace cbg {

template <int FMT> struct Launcher {
    static void dot(int arith, int grid, cudaStream_t s, const DotArgs& a);
    static void axpy(int arith, int epi, int grid, cudaStream_t s, const AxpyArgs& a);
    // bulk-copy pipelined DF32 dot (one block per SM)
    static void dot_tma(int grid, cudaStream_t s, const DotArgs& a, int* fault);
    static bool tma_fits();
    static void store(int grid, cudaStream_t s, const StoreArgs& a);
    static void spmv_code(int mode, int group, int grid, cudaStream_t s, const SpmvArgs& a);
    // per-step SpMV on the sliced-ELL copy (Arnoldi mode, double-float rows)
    static void spmv_sell(int grid, cudaStream_t s, const SellArgs& a);
    static void encode(int grid, cudaStream_t s, const double* v, long long n, unsigned char* codes,
                       EncParams ep);
    static void decode(int grid, cudaStream_t s, const unsigned char* codes, long long n, double scale,
                       double* out);
    static int occupancy_dot();
    static int occupancy_axpy();
    // resident blocks per SM of the per-step SpMV kernels of this code format (the CSR
    // Arnoldi kernel with one and 32 lanes per row, and the sliced-ELL kernel): the least
    static int occupancy_spmv();
    // batched persistent solve with thread-block clusters of `cluster` blocks
    static cudaError_t batched(int cluster, int grid, size_t smem, cudaStream_t s, const BatchArgs& a);
    static int batched_max_clusters(int cluster, size_t smem);
};

// SpMV with an FP64 input vector (residual, SPAI second stage, x += P t)
void spmv_f64(int mode, int group, int grid, cudaStream_t s, const SpmvArgs& a);
void spmv_sell_f64(int grid, cudaStream_t s, const SellArgs& a);
int spmv_occupancy();

}  // namespace cbg
