// multi_tc.cu -- multi-RHS basis product H = V^T W on the 5th-generation tensor cores
// (tcgen05) for the f16 basis, exact up to one rounding of W per 2048-row block.
//
// FP64-accurate products from FP16 tensor cores: both operands are cut into small exact
// integers ("digits"), every digit product is exact, and every FP32 accumulator stays an
// exact integer, so the tensor core computes integer dot products without error.
//  * V: a stored f16 code v (|v| <= 1 for a normalised basis vector, a multiple of 2^-24)
//    is the integer x = v 2^24, |x| <= 2^24, written as x = d0 + d1 2^11 + d2 2^22 with
//    signed digits |d_a| <= 1024 (exact in FP16).
//  * W: per vector r and block of KB = 2048 rows, with E_rb the exponent of the block's
//    largest |w| (|w| < 2^E_rb), the integer y = rint(w 2^(54 - E_rb)) (the only
//    rounding: relative 2^-55 of the block maximum) is cut into 14 signed base-16 digits
//    |e_b| <= 8, placed side by side in the N dimension (n = 14 r + b, N = 128).
//  * Products |d e| <= 2^13 and KB = 2048 rows keep each FP32 accumulator <= 2^24.
// One CTA per SM, 512 threads.  Per chunk of KC = 64 rows the threads write the digit
// planes of V (3 x 128 columns x 64 rows) and W (128 x 64) into shared memory in the
// canonical K-major layout (8-row x 16-byte core matrices), thread 0 issues 3 x 4
// tcgen05.mma (M = 128, N = 128, K = 16, FP16 x FP16 -> FP32 in tensor memory, one
// accumulator per V digit) and commits them to an mbarrier; chunks alternate between two
// buffers so the next chunk is cut while the tensor core works.  After every K block the
// four warps drain their 32 TMEM lanes (one basis column per lane) and combine the
// 3 x 14 digit sums per vector in double-float with the block's power-of-two scales.
// Every wait is bounded: a pipeline that stops making progress records a fault and
// the kernel leaves after freeing its tensor memory.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>

#include "../../include/cbgmres.h"
#include "cbg_kernels.cuh"
#include "cbg_tma.cuh"

using namespace cbg;

namespace {

constexpr int TC_THREADS = 512;          // 16 warps cut digits; warps 0-3 also drain TMEM
constexpr int TC_M = 128;                 // basis columns per CTA tile (TMEM lanes)
constexpr int TC_N = 128;                 // 8 vectors x 14 digits, padded
constexpr int KC = 64;                    // rows per chunk
constexpr int KB = 2048;                  // rows per exact accumulation block
constexpr int SV = 3;                     // digits of a V code
constexpr int SW = 14;                    // digits of a W entry
constexpr int WBITS = 4;                  // bits per W digit
constexpr int VBITS = 11;                 // bits per V digit
// |y| = |w| 2^(WSHIFT - E) < 2^54 stays inside the range of 14 signed base-16 digits
// (largest positive 7 (16^14 - 1) / 15 > 2^54)
constexpr int WSHIFT = 54;
constexpr int A_PLANE = TC_M * KC * 2;    // bytes of one V digit plane (16 KiB)
constexpr int B_PLANE = TC_N * KC * 2;    // bytes of the W digit plane (16 KiB)
constexpr int BUF = SV * A_PLANE + B_PLANE;
constexpr int TC_SMEM = 2 * BUF + 1024;   // two chunk buffers (+ alignment slack)
constexpr int SBO = (KC / 8) * 128;       // byte offset between 8-row core-matrix groups
constexpr int LBO = 128;                  // byte offset between K-adjacent core matrices
constexpr int TMEM_COLS = 512;            // 3 accumulators x 128 columns, rounded up

struct TcArgs {
    const unsigned short* V;  // f16 codes, column c at V + c * ld
    long long ld;
    int ncols;                // <= 128
    const double* scales;     // device [ncols]
    const double* W;          // n x k, column-major, leading dimension ldw
    long long ldw;
    long long n;
    int k;                    // <= 8
    const int* wexp;          // [nblk][8]: E_rb
    double* part;             // [gridDim.x][128][8]
    unsigned int* counter;
    double* H;                // [ncols][k]
    int* fault;
};

// byte offset of element (row m, k) in a K-major no-swizzle tile with 64 K-columns
__device__ __forceinline__ int kmaj_off(int m, int kk)
{
    return (m >> 3) * SBO + (kk >> 3) * LBO + (m & 7) * 16 + (kk & 7) * 2;
}

__device__ __forceinline__ uint64_t smem_desc(const void* p)
{
    uint64_t d = (uint64_t)((smem_addr(p) >> 4) & 0x3FFF);
    d |= (uint64_t)((LBO >> 4) & 0x3FFF) << 16;
    d |= (uint64_t)((SBO >> 4) & 0x3FFF) << 32;
    d |= (uint64_t)1 << 46;                     // descriptor version (sm_100 family)
    return d;                                   // no swizzle, base offset 0
}

__device__ __forceinline__ void mma_f16(uint32_t tmem, uint64_t da, uint64_t db, uint32_t idesc, int acc)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem),
        "l"(da), "l"(db), "r"(idesc), "r"(acc)
        : "memory");
}

__device__ __forceinline__ void mma_commit(uint64_t* bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                     smem_addr(bar))
                 : "memory");
}

// 32 consecutive TMEM columns of this warp's 32 lanes
__device__ __forceinline__ void tmem_ld32(uint32_t addr, float* v)
{
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(addr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 32; i++) v[i] = __uint_as_float(r[i]);
}

// signed digit of x in base 2^bits (|d| <= 2^(bits-1)), x <- (x - d) / 2^bits
__device__ __forceinline__ float next_digit(float& x, float base, float inv_base)
{
    const float q = rintf(x * inv_base);
    const float d = __fmaf_rn(-q, base, x);
    x = q;
    return d;
}

// per vector and KB-row block: E with max |w| < 2^E (the exponent of frexp)
__global__ void k_wexp(const double* W, long long ldw, long long n, int k, long long nblk, int* wexp)
{
    const long long total = nblk * 8;
    for (long long t = (long long)blockIdx.x * blockDim.y + threadIdx.y; t < total; t += (long long)gridDim.x * blockDim.y) {
        const long long b = t / 8;
        const int r = (int)(t - b * 8);
        unsigned long long mb = 0;
        if (r < k) {
            const long long i1 = (b + 1) * KB < n ? (b + 1) * KB : n;
            for (long long i = b * KB + threadIdx.x; i < i1; i += 32) {
                const unsigned long long u = (unsigned long long)__double_as_longlong(W[r * ldw + i]) & 0x7FFFFFFFFFFFFFFFull;
                mb = u > mb ? u : mb;
            }
        }
        for (int o = 16; o; o >>= 1) {
            const unsigned long long v = __shfl_xor_sync(0xffffffffu, mb, o);
            mb = v > mb ? v : mb;
        }
        if (threadIdx.x == 0) {
            int e = 0;
            if (mb) frexp(__longlong_as_double((long long)mb), &e);
            wexp[t] = e;
        }
    }
}

__global__ void __launch_bounds__(TC_THREADS, 1) k_dot_multi_tc(TcArgs a)
{
    extern __shared__ unsigned char tc_raw[];
    unsigned char* sm = reinterpret_cast<unsigned char*>(((size_t)tc_raw + 1023) & ~(size_t)1023);
    __shared__ __align__(8) uint64_t mbar[2];
    __shared__ uint32_t tbase;
    // A wait that timed out is recorded in flag[dp & 1] before the barrier of decision
    // point dp and read by everyone after it; alternating flags keep a fast warp's write
    // for the next decision point away from a slow warp's read of this one.
    __shared__ int flag[2];
    int dp = 0;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const long long nblk = (a.n + KB - 1) / KB;
    const long long bb = (long long)blockIdx.x * nblk / gridDim.x;       // this CTA's K blocks
    const long long be = ((long long)blockIdx.x + 1) * nblk / gridDim.x;

    // zero both buffers once: padding columns (ncols..127, vector digits 112..127) stay zero
    for (int i = tid; i < 2 * BUF / 16; i += TC_THREADS) reinterpret_cast<uint4*>(sm)[i] = make_uint4(0, 0, 0, 0);
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(&tbase)),
                     "r"(TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        flag[0] = 0;
        flag[1] = 0;
        mbar_init(&mbar[0], 1);
        mbar_init(&mbar[1], 1);
        mbar_init_fence();
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tbase;
    const uint32_t idesc = (1u << 4) | ((uint32_t)(TC_N >> 3) << 17) | ((uint32_t)(TC_M >> 4) << 24);

    // FP64 accumulators of this thread's column (TMEM lane = column) per vector
    double acc[8];
#pragma unroll
    for (int r = 0; r < 8; r++) acc[r] = 0.0;
    unsigned issued[2] = {0u, 0u};          // commits per buffer (phase tracking)

    // Each thread's inputs of a chunk (two 16-byte code groups of one column, one entry of
    // W) are loaded one chunk ahead, so their latency hides behind the current chunk.
    const int vc = warp * 8 + (lane & 7);
    const bool vlive = vc < a.ncols;
    const int wr = tid >> 6, wrow = tid & 63;
    auto load_chunk = [&](long long r0, uint4* raw, double& wv) {
        const unsigned short* col = a.V + (long long)vc * a.ld + r0;
#pragma unroll
        for (int p = 0; p < 2; p++) {
            const int g = (lane >> 3) + 4 * p;
            raw[p] = vlive ? __ldcs(reinterpret_cast<const uint4*>(col + g * 8)) : make_uint4(0, 0, 0, 0);
        }
        wv = (wr < a.k && r0 + wrow < a.n) ? __ldcs(a.W + wr * a.ldw + r0 + wrow) : 0.0;
    };
    uint4 nraw[2];
    double nw = 0.0;
    if (bb < be) load_chunk(bb * KB, nraw, nw);

    for (long long blk = bb; blk < be; blk++) {
        const long long row_b = blk * KB;
        const int nck = (int)((min((long long)KB, a.n - row_b) + KC - 1) / KC);
        int ew[8];
#pragma unroll
        for (int r = 0; r < 8; r++) ew[r] = a.wexp[blk * 8 + r];
        for (int ck = 0; ck < nck; ck++) {
            const int buf = ck & 1;
            unsigned char* A = sm + buf * BUF;
            unsigned char* Bm = A + SV * A_PLANE;
            // the MMAs that last read this buffer must be done (a timeout is recorded; the
            // block-wide decision to stop is taken after the barrier below)
            if (issued[buf] > 0 && !warp_wait(&mbar[buf], (issued[buf] - 1) & 1)) flag[dp & 1] = 1;
            const long long r0 = row_b + (long long)ck * KC;
            uint4 raw[2] = {nraw[0], nraw[1]};
            const double wcur = nw;
            {   // prefetch the next chunk (this block's next, or the next block's first)
                const long long rn = ck + 1 < nck ? r0 + KC : (blk + 1 < be ? (blk + 1) * KB : -1);
                if (rn >= 0) load_chunk(rn, nraw, nw);
            }
            // ---- V digits: warp w cuts columns 8w .. 8w+7; lane = column (lane & 7) and 8-row
            // groups (lane >> 3) + 4p, so the 32 lanes store 512 contiguous bytes of a plane
            if (!flag[dp & 1]) {
                const int c = vc;
#pragma unroll
                for (int p = 0; p < 2; p++) {
                    const int g = (lane >> 3) + 4 * p;
                    const unsigned int w4[4] = {raw[p].x, raw[p].y, raw[p].z, raw[p].w};
                    unsigned int out[SV][4];
#pragma unroll
                    for (int h = 0; h < 4; h++) {
                        float x0 = dec_f16(w4[h] & 0xFFFFu) * 16777216.0f, x1 = dec_f16(w4[h] >> 16) * 16777216.0f;
                        float d0[SV], d1[SV];
#pragma unroll
                        for (int sd = 0; sd < SV; sd++) {
                            d0[sd] = next_digit(x0, 2048.0f, 1.0f / 2048.0f);
                            d1[sd] = next_digit(x1, 2048.0f, 1.0f / 2048.0f);
                        }
#pragma unroll
                        for (int sd = 0; sd < SV; sd++) {
                            const __half2 hp = __floats2half2_rn(d0[sd], d1[sd]);
                            out[sd][h] = *reinterpret_cast<const unsigned int*>(&hp);
                        }
                    }
#pragma unroll
                    for (int sd = 0; sd < SV; sd++)
                        *reinterpret_cast<uint4*>(A + sd * A_PLANE + kmaj_off(c, g * 8)) =
                            make_uint4(out[sd][0], out[sd][1], out[sd][2], out[sd][3]);
                }
            }
            // ---- W digits: thread t takes vector t / 64 and row t % 64 of the chunk; the
            // scaled integer y = rint(w 2^(54 - E)) comes from w's bits (no FP64 arithmetic)
            if (!flag[dp & 1]) {
                const int r = wr, row = wrow;
                if (r < a.k) {
                    long long y = 0;
                    {
                        const unsigned long long u = (unsigned long long)__double_as_longlong(wcur);
                        const int ex = (int)((u >> 52) & 0x7FF);
                        if (ex > 0) {   // zero and subnormal inputs (below 2^-1022) contribute nothing
                            const unsigned long long m = (u & 0xFFFFFFFFFFFFFull) | (1ull << 52);
                            // w = m 2^(ex - 1075), |w| < 2^E gives ex <= E + 1022, so
                            // y = m 2^(ex - 1021 - E) = m 2^-sh with sh >= -1 (|y| < 2^54)
                            const int sh = ew[r] + 1021 - ex;
                            unsigned long long q = 0;
                            if (sh <= 0) {
                                q = m << (-sh);
                            } else if (sh < 64) {   // round to nearest, ties to even
                                q = m >> sh;
                                const unsigned long long rem = m & ((1ull << sh) - 1), half = 1ull << (sh - 1);
                                if (rem > half || (rem == half && (q & 1ull))) q++;
                            }
                            y = (u >> 63) ? -(long long)q : (long long)q;
                        }
                    }
                    unsigned short* Bh = reinterpret_cast<unsigned short*>(Bm);
#pragma unroll
                    for (int bd = 0; bd < SW; bd++) {
                        const long long t = ((y + 8) & 15) - 8;
                        y = (y - t) >> 4;
                        Bh[kmaj_off(r * SW + bd, row) >> 1] = __half_as_ushort(__int2half_rn((int)t));
                    }
                }
            }
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            __syncthreads();
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            if (flag[dp++ & 1]) break;          // uniform: every thread passed the barrier
            if (tid == 0) {
#pragma unroll
                for (int s = 0; s < SV; s++) {
#pragma unroll
                    for (int kk = 0; kk < KC / 16; kk++) {
                        const uint64_t da = smem_desc(A + s * A_PLANE + kk * 2 * LBO);
                        const uint64_t db = smem_desc(Bm + kk * 2 * LBO);
                        mma_f16(tmem + (uint32_t)(s * TC_N), da, db, idesc, (ck > 0 || kk > 0) ? 1 : 0);
                    }
                }
                mma_commit(&mbar[buf]);
            }
            issued[buf]++;
        }
        if (flag[(dp - 1) & 1]) break;      // the chunk loop stopped at a failed decision point
        // ---- drain: the last chunk's commit covers every MMA of the block
        {
            const int lb = (nck - 1) & 1;
            if (!warp_wait(&mbar[lb], (issued[lb] - 1) & 1)) flag[dp & 1] = 1;
        }
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncthreads();
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        if (flag[dp++ & 1]) break;
        // digit sums x 2^(11 s + 4 b): exact FP32 values below 2^99, summed per vector in
        // double-float, then scaled by the block's 2^(E_rb - 54 - 24) in FP64 (warps 0-3:
        // warp w reads TMEM lanes 32w .. 32w+31, i.e. basis columns 32w + lane)
        if (warp < 4) {
        float ds[8], dc[8];
#pragma unroll
        for (int r = 0; r < 8; r++) { ds[r] = 0.f; dc[r] = 0.f; }
#pragma unroll 1
        for (int s = 0; s < SV; s++) {
#pragma unroll 1
            for (int q = 0; q < TC_N / 32; q++) {
                float v[32];
                tmem_ld32(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(s * TC_N + q * 32), v);
#pragma unroll
                for (int i = 0; i < 32; i++) {
                    const int nidx = q * 32 + i, r = nidx / SW, b = nidx - r * SW;
                    if (r < 8) df_add(ds[r], dc[r], ldexpf(v[i], VBITS * s + WBITS * b), 0.f);
                }
            }
        }
#pragma unroll
        for (int r = 0; r < 8; r++) acc[r] = __fma_rn(df_to_double(ds[r], dc[r]), ldexp(1.0, ew[r] - WSHIFT - 24), acc[r]);
        }
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncthreads();                    // drained before the next block's first MMA overwrites
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    }
    // drain outstanding commits before freeing tensor memory (bounded)
    for (int b2 = 0; b2 < 2; b2++)
        if (issued[b2] > 0) warp_wait(&mbar[b2], (issued[b2] - 1) & 1);
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS) : "memory");
    if ((flag[0] | flag[1]) && tid == 0 && a.fault) atomicExch(a.fault, 1);
    // per-CTA partials, then the last CTA adds them in a fixed order
    if (tid < TC_M) {
#pragma unroll
        for (int r = 0; r < 8; r++) a.part[((long long)blockIdx.x * TC_M + tid) * 8 + r] = acc[r];
    }
    if (last_block(a.counter)) {
        for (int i = warp; i < a.ncols * a.k; i += TC_THREADS / 32) {
            const int col = i / a.k, r = i - col * a.k;
            double sum = 0.0;
            for (unsigned int b = lane; b < gridDim.x; b += 32) sum += __ldcg(a.part + ((long long)b * TC_M + col) * 8 + r);
            sum = warp_sum(sum);
            if (lane == 0) a.H[i] = sum * a.scales[col];
        }
    }
}

int tc_grid()
{
    int dev = 0, sms = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return std::max(1, sms);
}

}  // namespace

// Tensor-core multi-RHS product for the f16 basis (ncols <= 128, k <= 8).  Workspace
// layout: [counter, fault | wexp | partials].
size_t cbg_tc_multi_workspace(int64_t ld)
{
    const long long nblk = (ld + KB - 1) / KB;
    return 256 + ((size_t)nblk * 8 * sizeof(int) + 255) / 256 * 256 + (size_t)tc_grid() * TC_M * 8 * sizeof(double);
}

int cbg_tc_multi(int64_t n, int ncols, const void* V, int64_t ld, const double* scales, int k, const double* W,
                 int64_t ldw, double* H, void* workspace, cudaStream_t s, int** fault_out)
{
    unsigned char* ws = static_cast<unsigned char*>(workspace);
    unsigned int* counter = reinterpret_cast<unsigned int*>(ws);
    int* fault = reinterpret_cast<int*>(ws + 4);
    const long long nblk = (n + KB - 1) / KB;
    int* wexp = reinterpret_cast<int*>(ws + 256);
    double* part = reinterpret_cast<double*>(ws + 256 + ((size_t)((ld + KB - 1) / KB) * 8 * sizeof(int) + 255) / 256 * 256);
    if (fault_out) *fault_out = fault;
    if (cudaMemsetAsync(ws, 0, 8, s) != cudaSuccess) return CBG_ERR_CUDA;
    k_wexp<<<(int)std::min<long long>((nblk * 8 + 7) / 8, 4096), dim3(32, 8), 0, s>>>(W, ldw, n, k, nblk, wexp);
    static const bool attr = [] {
        cudaFuncSetAttribute(k_dot_multi_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, TC_SMEM);
        return true;
    }();
    (void)attr;
    TcArgs a{};
    a.V = static_cast<const unsigned short*>(V);
    a.ld = ld;
    a.ncols = ncols;
    a.scales = scales;
    a.W = W;
    a.ldw = ldw;
    a.n = n;
    a.k = k;
    a.wexp = wexp;
    a.part = part;
    a.counter = counter;
    a.H = H;
    a.fault = fault;
    k_dot_multi_tc<<<tc_grid(), TC_THREADS, TC_SMEM, s>>>(a);
    return cudaGetLastError() == cudaSuccess ? CBG_OK : CBG_ERR_CUDA;
}
