// cbg_launch_impl.cuh -- definitions of the launchers declared in cbg_launch.h.
#pragma once
#include <algorithm>

#include "cbg_launch.h"

namespace cbg {

#define CBG_SPMV_GROUPS(XF, MODE)                                                              \
    switch (group) {                                                                           \
    case 1: k_spmv<XF, 1, MODE><<<grid, THREADS, 0, s>>>(a); break;                            \
    case 2: k_spmv<XF, 2, MODE><<<grid, THREADS, 0, s>>>(a); break;                            \
    case 4: k_spmv<XF, 4, MODE><<<grid, THREADS, 0, s>>>(a); break;                            \
    case 8: k_spmv<XF, 8, MODE><<<grid, THREADS, 0, s>>>(a); break;                            \
    case 16: k_spmv<XF, 16, MODE><<<grid, THREADS, 0, s>>>(a); break;                          \
    default: k_spmv<XF, 32, MODE><<<grid, THREADS, 0, s>>>(a); break;                          \
    }

template <int FMT> void Launcher<FMT>::dot(int arith, int grid, cudaStream_t s, const DotArgs& a)
{
    if (arith == ARITH_DF32) k_basis_dot<FMT, ARITH_DF32><<<grid, THREADS, 0, s>>>(a);
    else k_basis_dot<FMT, ARITH_FP64><<<grid, THREADS, 0, s>>>(a);
}

template <int FMT>
void Launcher<FMT>::axpy(int arith, int epi, int grid, cudaStream_t s, const AxpyArgs& a)
{
    if (arith == ARITH_DF32) {
        if (epi == EPI_SUB) k_basis_axpy<FMT, ARITH_DF32, EPI_SUB><<<grid, THREADS, 0, s>>>(a);
        else if (epi == EPI_XUPD) k_basis_axpy<FMT, ARITH_DF32, EPI_XUPD><<<grid, THREADS, 0, s>>>(a);
        else k_basis_axpy<FMT, ARITH_DF32, EPI_PLAIN><<<grid, THREADS, 0, s>>>(a);
    } else {
        if (epi == EPI_SUB) k_basis_axpy<FMT, ARITH_FP64, EPI_SUB><<<grid, THREADS, 0, s>>>(a);
        else if (epi == EPI_XUPD) k_basis_axpy<FMT, ARITH_FP64, EPI_XUPD><<<grid, THREADS, 0, s>>>(a);
        else k_basis_axpy<FMT, ARITH_FP64, EPI_PLAIN><<<grid, THREADS, 0, s>>>(a);
    }
}

// Ring stages of the pipelined dot: the opt-in shared memory left by the kernel's static
// shared memory (queried once per process), and the matching opt-in attribute.
struct TmaPlan {
    int stages = 0;
    size_t smem = 0;
};
template <int FMT> static const TmaPlan& tma_plan()
{
    static const TmaPlan plan = [] {
        using G = TmaGeom<FMT>;
        TmaPlan p;
        cudaFuncAttributes fa{};
        const int static_bytes =
            cudaFuncGetAttributes(&fa, k_basis_dot_tma<FMT>) == cudaSuccess ? (int)fa.sharedSizeBytes : TMA_SMEM_OPTIN;
        p.stages = tma_stages(G::STAGE_DOT, static_bytes);
        p.smem = tma_smem_bytes(p.stages, G::STAGE_DOT);
        if (p.stages >= 2)
            cudaFuncSetAttribute(k_basis_dot_tma<FMT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)p.smem);
        return p;
    }();
    return plan;
}

template <int FMT> bool Launcher<FMT>::tma_fits() { return tma_plan<FMT>().stages >= 2; }

template <int FMT> void Launcher<FMT>::dot_tma(int grid, cudaStream_t s, const DotArgs& a, int* fault)
{
    // cooperative: the kernel's blocks meet at a grid barrier before the cross-block sum
    const TmaPlan& p = tma_plan<FMT>();
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(DOT_THREADS);
    cfg.dynamicSmemBytes = p.smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    cudaLaunchKernelEx(&cfg, k_basis_dot_tma<FMT>, a, p.stages, fault);
}

template <int FMT> void Launcher<FMT>::store(int grid, cudaStream_t s, const StoreArgs& a)
{
    // mode 0: at least two blocks (block 0 runs the Givens update, the others encode)
    k_store<FMT><<<a.mode == 0 ? (grid > 1 ? grid : 2) : grid, THREADS, 0, s>>>(a);
}

template <int FMT>
void Launcher<FMT>::spmv_code(int mode, int group, int grid, cudaStream_t s, const SpmvArgs& a)
{
    if (mode == SPMV_ARNOLDI) { CBG_SPMV_GROUPS(FMT, SPMV_ARNOLDI) }
    else { CBG_SPMV_GROUPS(FMT, SPMV_PLAIN) }
}

template <int FMT> void Launcher<FMT>::spmv_sell(int grid, cudaStream_t s, const SellArgs& a)
{
    k_spmv_sell<FMT><<<grid, THREADS, 0, s>>>(a);
}

template <int FMT>
void Launcher<FMT>::encode(int grid, cudaStream_t s, const double* v, long long n, unsigned char* codes,
                           EncParams ep)
{
    k_encode_vec<FMT><<<grid, THREADS, 0, s>>>(v, n, codes, ep);
}

template <int FMT>
void Launcher<FMT>::decode(int grid, cudaStream_t s, const unsigned char* codes, long long n, double scale,
                           double* out)
{
    k_decode_vec<FMT><<<grid, THREADS, 0, s>>>(codes, n, scale, out);
}

template <int FMT> int Launcher<FMT>::occupancy_dot()
{
    int b = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_basis_dot<FMT, ARITH_DF32>, THREADS, 0);
    return b;
}

template <int FMT> int Launcher<FMT>::occupancy_axpy()
{
    int b = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_basis_axpy<FMT, ARITH_DF32, EPI_SUB>, THREADS, 0);
    return b;
}

template <int FMT> int Launcher<FMT>::occupancy_spmv()
{
    int b1 = 0, b32 = 0, bs = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b1, k_spmv<FMT, 1, SPMV_ARNOLDI>, THREADS, 0);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b32, k_spmv<FMT, 32, SPMV_ARNOLDI>, THREADS, 0);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bs, k_spmv_sell<FMT>, THREADS, 0);
    return std::min(b1, std::min(b32, bs));
}

}  // namespace cbg

namespace cbg {

template <int FMT> static void batched_opt_in(size_t smem)
{
    cudaFuncSetAttribute(k_batched<FMT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    cudaFuncSetAttribute(k_batched<FMT>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
}

template <int FMT>
cudaError_t Launcher<FMT>::batched(int cluster, int grid, size_t smem, cudaStream_t s, const BatchArgs& a)
{
    batched_opt_in<FMT>(smem);
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(BT_THREADS);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = cluster;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k_batched<FMT>, a);
}

template <int FMT> int Launcher<FMT>::batched_max_clusters(int cluster, size_t smem)
{
    batched_opt_in<FMT>(smem);
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(cluster);
    cfg.blockDim = dim3(BT_THREADS);
    cfg.dynamicSmemBytes = smem;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = cluster;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int n = 0;
    if (cudaOccupancyMaxActiveClusters(&n, k_batched<FMT>, &cfg) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return n;
}

}  // namespace cbg
