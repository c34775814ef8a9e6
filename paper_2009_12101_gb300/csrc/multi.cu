// multi.cu -- multi-RHS basis product H = V^T W for k vectors that share one compressed
// basis (the orthogonalisation of block Krylov methods; the paper has no counterpart:
// its GMRES has one right-hand side).
//
// Reading V once for all k vectors turns the k basis GEMVs into one split-K GEMM whose
// arithmetic (DF32, as in the single-vector kernels) dominates for k > 2.  Each block
// owns a contiguous range of row tiles (TR = 1024 rows).  Per tile it stages W's rows
// (already split into FP32 hi / lo planes) in shared memory; warp w then takes column
// groups w, w+8, ... of CG = 32/KR columns: lane l takes rows l, l+32, ... (so a warp
// reads 32 consecutive codes of a column, and its rows of W from shared memory without
// bank conflicts) and keeps CG x KR double-float accumulators (pairs of right-hand sides
// on the packed FP32x2 pipe).  At the end of a tile the warp folds the 32 accumulators
// with the transposing butterfly (every lane ends with one (column, vector) total) and
// adds it to the block's FP64 totals in shared memory; a (column, vector) pair always
// belongs to the same warp, so the sums are deterministic.  Blocks leave per-column
// partials and the last block adds them in a fixed order.
#include <cuda_runtime.h>

#include <algorithm>
#include <type_traits>

#include "../../include/cbgmres.h"
#include "cbg_kernels.cuh"

using namespace cbg;

void cbg_record_cuda_error(cudaError_t e);   // solver.cu
size_t cbg_tc_multi_workspace(int64_t ld);   // multi_tc.cu
int cbg_tc_multi(int64_t n, int ncols, const void* V, int64_t ld, const double* scales, int k, int ldh, const double* W,
                 int64_t ldw, double* H, void* workspace, cudaStream_t s, int** fault_out);

namespace {

constexpr int MT = 256;              // threads per block
constexpr int MNW = MT / 32;
constexpr int TR = 1024;             // rows per tile
constexpr int KMAX = 8;              // right-hand sides per launch
constexpr int KCALL = 64;            // right-hand sides per call (groups of KMAX)

struct MultiArgs {
    const unsigned char* V;
    long long ldb;            // bytes per basis column
    int ncols;
    const double* scales;     // device [ncols]
    const float* wsplit;      // W split: hi[KR][ld], then lo[KR][ld]
    long long ld;             // rows per column (multiple of TILE_ROWS)
    double* part;             // [gridDim.x][ncols][KR]
    unsigned int* counter;
    double* H;                // [ncols][k] (row-major), device
    int k;                    // vectors actually requested (<= KR)
    int ldh;                  // row stride of H (>= k)
};

// W (n x k, column-major, leading dimension ldw) -> hi / lo FP32 planes of KR x ld, zero
// beyond n and beyond k
__global__ void k_split_multi(const double* W, long long ldw, long long n, long long ld, int k, int KR, float* out)
{
    const long long total = (long long)KR * ld;
    for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (long long)gridDim.x * blockDim.x) {
        const long long r = t / ld, i = t - r * ld;
        float h = 0.f, l = 0.f;
        if (r < k && i < n) split_f64(W[r * ldw + i], h, l);
        out[t] = h;
        out[total + t] = l;
    }
}

// one code of a basis column, read as its storage word, and its exact FP32 (pair) value
template <int FMT> struct Code {
    using T = typename std::conditional<FmtInfo<FMT>::bytes == 8, unsigned long long,
              typename std::conditional<FmtInfo<FMT>::bytes == 4, unsigned int,
              typename std::conditional<FmtInfo<FMT>::bytes == 2, unsigned short, unsigned char>::type>::type>::type;
    static __device__ __forceinline__ T load(const unsigned char* col, long long row)
    {
        return __ldcs(reinterpret_cast<const T*>(col) + row);
    }
    static __device__ __forceinline__ void value(T c, float& hi, float& lo)
    {
        lo = 0.f;
        if constexpr (FMT == F64) split_f64(__longlong_as_double((long long)c), hi, lo);
        else if constexpr (FMT == F32) hi = __uint_as_float(c);
        else if constexpr (FMT == F16) hi = dec_f16(c);
        else if constexpr (FMT == BF16) hi = dec_bf16(c);
        else if constexpr (FMT == E4M3) { float b; dec_e4m3x2(c, hi, b); }
        else if constexpr (FMT == I32) dec_i32((int)c, hi, lo);
        else hi = dec_i16((int)(short)c);
    }
};

template <int FMT, int KR>
__global__ void __launch_bounds__(MT, 1) k_dot_multi(MultiArgs a)
{
    using CT = Code<FMT>;
    constexpr int CODE_REGS = 32 / KR * (FmtInfo<FMT>::bytes == 8 ? 2 : 1);
    constexpr int EE = 32 / CODE_REGS < 8 ? (32 / CODE_REGS > 0 ? 32 / CODE_REGS : 1) : 8;   // rows per lane and step, 32 apart
    constexpr int CG = 32 / KR;                // columns per warp group (CG x KR = 32 sums)
    constexpr int STEPS = TR / (32 * EE);      // warp steps per tile
    extern __shared__ __align__(16) float msm[];
    float* wh_s = msm;                         // [KR][TR]
    float* wl_s = msm + KR * TR;               // [KR][TR]
    __shared__ double tot[MAXCOLS * KMAX];     // block totals [col][KR]
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int ncols = a.ncols;
    const int ngroups = (ncols + CG - 1) / CG;
    const long long ntiles = a.ld / TR;
    const long long tb = (long long)blockIdx.x * ntiles / gridDim.x;
    const long long te = ((long long)blockIdx.x + 1) * ntiles / gridDim.x;
    for (int i = threadIdx.x; i < ncols * KR; i += MT) tot[i] = 0.0;

    for (long long t = tb; t < te; t++) {
        const long long r0 = t * TR;
        __syncthreads();                       // previous tile's W no longer read
        for (int i = threadIdx.x; i < KR * TR / 4; i += MT) {
            const int r = i / (TR / 4), c = i - r * (TR / 4);
            reinterpret_cast<float4*>(wh_s)[i] =
                __ldcg(reinterpret_cast<const float4*>(a.wsplit + (long long)r * a.ld + r0) + c);
            reinterpret_cast<float4*>(wl_s)[i] =
                __ldcg(reinterpret_cast<const float4*>(a.wsplit + (long long)(KR + r) * a.ld + r0) + c);
        }
        __syncthreads();
        for (int g = warp; g < ngroups; g += MNW) {
            const int c0 = g * CG;
            float2 S2[CG * KR / 2], C2[CG * KR / 2];   // index q * KR/2 + r/2: column q, vectors (r, r+1)
#pragma unroll
            for (int i = 0; i < CG * KR / 2; i++) { S2[i] = make_float2(0.f, 0.f); C2[i] = make_float2(0.f, 0.f); }
            for (int st = 0; st < STEPS; st++) {
                const int rb = st * 32 * EE + lane;      // rows rb + 32 e of the tile
                // all codes of the step in flight at once
                typename CT::T code[EE][CG];
#pragma unroll
                for (int e = 0; e < EE; e++)
#pragma unroll
                    for (int q = 0; q < CG; q++)
                        code[e][q] = c0 + q < ncols ? CT::load(a.V + (long long)(c0 + q) * a.ldb, r0 + rb + 32 * e)
                                                    : (typename CT::T)0;
#pragma unroll
                for (int e = 0; e < EE; e++) {
                    float wh[KR], wl[KR];
#pragma unroll
                    for (int r = 0; r < KR; r++) {
                        wh[r] = wh_s[r * TR + rb + 32 * e];
                        wl[r] = wl_s[r * TR + rb + 32 * e];
                    }
#pragma unroll
                    for (int q = 0; q < CG; q++) {
                        float vh, vl;
                        CT::value(code[e][q], vh, vl);
#pragma unroll
                        for (int r = 0; r < KR; r += 2) {
                            const float2 w2 = make_float2(wh[r], wh[r + 1]);
                            const float2 nw2 = make_float2(-wh[r], -wh[r + 1]);
                            const float2 l2 = make_float2(wl[r], wl[r + 1]);
                            if constexpr (SingleFloat<FMT>::value)
                                df2_mac(S2[q * KR / 2 + r / 2], C2[q * KR / 2 + r / 2], make_float2(vh, vh), w2, nw2, l2);
                            else
                                df2_mac2(S2[q * KR / 2 + r / 2], C2[q * KR / 2 + r / 2], make_float2(vh, vh),
                                         make_float2(vl, vl), w2, nw2, l2);
                        }
                    }
                }
#pragma unroll
                for (int i = 0; i < CG * KR / 2; i++) df2_renorm(S2[i], C2[i]);
            }
            // 32 sums per lane -> one (column, vector) total per lane
            float S[32], C[32];
#pragma unroll
            for (int i = 0; i < 16; i++) {
                S[2 * i] = S2[i].x; S[2 * i + 1] = S2[i].y;
                C[2 * i] = C2[i].x; C[2 * i + 1] = C2[i].y;
            }
            const int idx = df_warp_fold<32>(S, C, lane);   // = q * KR + r
            const int q = idx / KR, r = idx - q * KR;
            if (c0 + q < ncols) tot[(c0 + q) * KR + r] += df_to_double(S[0], C[0]);
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < ncols * KR; i += MT) a.part[(long long)blockIdx.x * ncols * KR + i] = tot[i];
    if (last_block(a.counter))   // items col * KR + r; the partials of r >= k are zero and not kept
        reduce_block_parts(a.part, (long long)ncols * KR, gridDim.x, ncols * KR, warp, MNW, [&](int i, double sum) {
            const int col = i / KR, r = i - col * KR;
            if (r < a.k) a.H[(long long)col * a.ldh + r] = sum * a.scales[col];
        });
}

template <int FMT, int KR> void launch_multi(int grid, cudaStream_t s, const MultiArgs& a)
{
    const size_t smem = (size_t)2 * KR * TR * sizeof(float);
    static const bool attr = [] {
        cudaFuncSetAttribute(k_dot_multi<FMT, KR>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)((size_t)2 * KR * TR * sizeof(float)));
        return true;
    }();
    (void)attr;
    k_dot_multi<FMT, KR><<<grid, MT, smem, s>>>(a);
}

template <int KR> void launch_fmt(int fmt, int grid, cudaStream_t s, const MultiArgs& a)
{
    switch (fmt) {
    case CBG_F64: launch_multi<F64, KR>(grid, s, a); break;
    case CBG_F32: launch_multi<F32, KR>(grid, s, a); break;
    case CBG_F16: launch_multi<F16, KR>(grid, s, a); break;
    case CBG_BF16: launch_multi<BF16, KR>(grid, s, a); break;
    case CBG_E4M3: launch_multi<E4M3, KR>(grid, s, a); break;
    case CBG_I32: launch_multi<I32, KR>(grid, s, a); break;
    default: launch_multi<I16, KR>(grid, s, a); break;
    }
}

int kr_for(int k) { return k <= 2 ? 2 : (k <= 4 ? 4 : 8); }
int multi_grid()
{
    int dev = 0, sms = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return 2 * std::max(1, sms);
}

// one group of k <= KMAX vectors: H[c * ldh + r]
int dot_multi_group(int fmt, int64_t n, int ncols, const void* V, int64_t ld, const double* scales, int k,
                    const double* W, int64_t ldw, double* H, int ldh, void* workspace, cudaStream_t s, bool tc)
{
    if (tc) {
        int rc = cbg_tc_multi(n, ncols, V, ld, scales, k, ldh, W, ldw, H, workspace, s, nullptr);
        if (rc) { cbg_record_cuda_error(cudaGetLastError()); return rc; }
        return CBG_OK;
    }
    const int KR = kr_for(k);
    unsigned char* ws = static_cast<unsigned char*>(workspace);
    unsigned int* counter = reinterpret_cast<unsigned int*>(ws);
    float* wsplit = reinterpret_cast<float*>(ws + 256);
    const size_t split = (size_t)2 * KR * ld * sizeof(float);
    double* part = reinterpret_cast<double*>(ws + 256 + (split + 255) / 256 * 256);
    cudaError_t e = cudaMemsetAsync(counter, 0, sizeof(unsigned int), s);
    if (e != cudaSuccess) { cbg_record_cuda_error(e); return CBG_ERR_CUDA; }
    const long long total = (long long)KR * ld;
    k_split_multi<<<(int)std::min<long long>((total + 255) / 256, 4096), 256, 0, s>>>(W, ldw, n, ld, k, KR, wsplit);
    MultiArgs a{};
    a.V = static_cast<const unsigned char*>(V);
    a.ldb = ld * cbgmres_format_bytes(fmt);
    a.ncols = ncols;
    a.scales = scales;
    a.wsplit = wsplit;
    a.ld = ld;
    a.part = part;
    a.counter = counter;
    a.H = H;
    a.k = k;
    a.ldh = ldh;
    const int grid = multi_grid();
    if (KR == 2) launch_fmt<2>(fmt, grid, s, a);
    else if (KR == 4) launch_fmt<4>(fmt, grid, s, a);
    else launch_fmt<8>(fmt, grid, s, a);
    e = cudaGetLastError();
    if (e != cudaSuccess) { cbg_record_cuda_error(e); return CBG_ERR_CUDA; }
    return CBG_OK;
}

}  // namespace

extern "C" {

size_t cbg_basis_dot_multi_workspace(int64_t ld, int ncols, int k)
{
    if (ld < 1 || ncols < 1 || ncols > MAXCOLS || k < 1 || k > KCALL) return 0;
    const int KR = kr_for(std::min(k, KMAX));
    const size_t split = (size_t)2 * KR * ld * sizeof(float);
    const size_t part = (size_t)multi_grid() * ncols * KR * sizeof(double);
    const size_t cuda_core = 256 + (split + 255) / 256 * 256 + (part + 255) / 256 * 256;
    return std::max(cuda_core, cbg_tc_multi_workspace(ld));
}

int cbg_basis_dot_multi_path(int fmt, int64_t n, int ncols, const void* V, int64_t ld, const double* scales, int k,
                             const double* W, int64_t ldw, double* H, void* workspace, size_t ws_bytes, void* stream,
                             int path)
{
    if (cbgmres_format_bytes(fmt) == 0 || n < 1 || ncols < 1 || ncols > MAXCOLS || k < 1 || k > KCALL || !V ||
        ld < n || ld % TILE_ROWS || !scales || !W || ldw < n || !H || !workspace ||
        ws_bytes < cbg_basis_dot_multi_workspace(ld, ncols, k) || path < 0 || path > 2)
        return CBG_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    const bool tc_ok = fmt == CBG_F16 && ncols <= 128;
    if (path == 2 && !tc_ok) return CBG_ERR_UNSUPPORTED;
    const bool tc = path == 2 || (path == 0 && tc_ok);
    // groups of up to KMAX vectors, one after the other on the stream (the workspace is reused)
    for (int r0 = 0; r0 < k; r0 += KMAX) {
        const int kg = std::min(KMAX, k - r0);
        int rc = dot_multi_group(fmt, n, ncols, V, ld, scales, kg, W + (long long)r0 * ldw, ldw, H + r0, k, workspace,
                                 s, tc);
        if (rc) return rc;
    }
    return CBG_OK;
}

int cbg_basis_dot_multi(int fmt, int64_t n, int ncols, const void* V, int64_t ld, const double* scales, int k,
                        const double* W, int64_t ldw, double* H, void* workspace, size_t ws_bytes, void* stream)
{
    return cbg_basis_dot_multi_path(fmt, n, ncols, V, ld, scales, k, W, ldw, H, workspace, ws_bytes, stream, 0);
}

}  // extern "C"
