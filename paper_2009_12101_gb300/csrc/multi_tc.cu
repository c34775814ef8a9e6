// multi_tc.cu -- multi-RHS basis product H = V^T W on the 5th-generation tensor cores
// (tcgen05) for the f16 basis, exact up to one truncation of W per 512-row block.
//
// FP64-accurate products from FP16 tensor cores: both operands are cut into small exact
// pieces ("digits"), every digit product is exact, and every FP32 accumulator stays on a
// grid of at most 2^24 points, so the tensor core adds without rounding.
//  * V: a stored f16 code v (|v| <= 1, the range of normalised basis vectors) is cut in
//    packed f16 arithmetic into v = hi 2^-11 + lo 2^-12 with an integer |hi| <= 2048 and
//    lo a multiple of 2^-12 with |lo| <= 1 (both exact in FP16).
//  * W: per vector r and block of KB = 512 rows, with E the exponent of the largest |w|
//    of the block (|w| < 2^E), the integer y = trunc(w 2^(54 - E)) (the only rounding:
//    below 2^-54 of the block maximum) is cut into 14 signed base-16 digits e_b in
//    [-8, 7].  The digits sit in the N dimension digit-major (n = 8 b + r', r' = r for
//    b < 8 and r xor 4 above, which makes the digit stores bank-conflict free).
//  * |hi e| <= 2^14 and |lo e| <= 2^15 grid points, so 512 rows stay within 2^24.
// One CTA per SM: 16 producer warps and one MMA warp.  Per chunk of KC = 64 rows the
// producers write the two V digit planes (128 columns x 64 rows) and the W digit plane
// (112 x 64) into shared memory in the canonical K-major layout (8-row x 16-byte core
// matrices) and arrive on the chunk buffer's "full" barrier; the MMA warp issues
// 2 x 4 tcgen05.mma (M = 128, N = 112, K = 16, FP16 x FP16 -> FP32 in tensor memory)
// and commits them to the buffer's "empty" barrier.  Three buffers let the producers run
// ahead of the tensor core; the inputs of chunk q + 2 are loaded into registers while
// chunk q is cut.  Tensor memory holds two accumulator sets (blocks alternate), so the
// sums of block p are read ("drained") by all producer warps during block p + 1, while
// the tensor core fills the other set.  A drain combines the 14 digit sums per vector in
// double-float (FP32 pairs) and adds them, scaled by 2^(E_p - Eref), to running
// double-float sums (Eref: the largest block exponent so far); FP64 is used only in the
// final cross-CTA reduction.  The block exponents are computed in the kernel one block
// ahead from the same W rows.  Every wait is bounded: a pipeline that stops making
// progress records a fault, the other warps see it and leave, and tensor memory is freed
// after the last MMA has completed.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>

#include "../../include/cbgmres.h"
#include "cbg_kernels.cuh"
#include "cbg_tma.cuh"

using namespace cbg;

namespace {

constexpr int PRODUCERS = 16;                 // warps that cut digits and drain
constexpr int MMA_WARP = PRODUCERS;           // the warp that issues the MMAs
constexpr int TC_THREADS = (PRODUCERS + 1) * 32;
constexpr int TC_M = 128;                     // basis columns per CTA tile (TMEM lanes)
constexpr int NVEC = 8;                       // right-hand sides per launch
constexpr int SW = 14;                        // digits of a W entry
constexpr int TC_N = SW * NVEC;               // 112
constexpr int KC = 64;                        // rows per chunk
constexpr int KB = 512;                       // rows per exact accumulation block
constexpr int CPB = KB / KC;                  // chunks per block
constexpr int SV = 2;                         // digit slices of a V code
constexpr int NBUF = 3;                       // chunk buffers
constexpr int WSHIFT = 54;                    // |y| = |w| 2^(WSHIFT - E) < 2^54
constexpr unsigned long long WBIAS = 0x0088888888888888ull;   // 8 in each of the 14 nibbles
constexpr int E_ZERO = -100000;               // block exponent of an all-zero block
constexpr int E_BAD = 100000;                 // ... of a block with an infinity or NaN
constexpr int DROP = 100;                     // sums below 2^-DROP of the running scale: dropped
constexpr int A_PLANE = TC_M * KC * 2;        // bytes of one V digit plane (16 KiB)
constexpr int B_ROWS = 128;                   // W digit plane rows: 112 used, 16 scratch
constexpr int B_PLANE = B_ROWS * KC * 2;      // 16 KiB
constexpr int BUF = SV * A_PLANE + B_PLANE;
constexpr int TC_SMEM = NBUF * BUF + 1024;    // chunk buffers (+ alignment slack)
constexpr int ROWB = KC * 2;                  // bytes of one operand row (64 K values)
constexpr int SBO = 8 * ROWB;                 // byte offset between 8-row groups
constexpr int TMEM_COLS = 512;                // 2 sets x 2 slices x 128 columns
constexpr int SET_COLS = 256;
constexpr int SLICE_COLS = 128;
constexpr unsigned int ABS_HI = 0x7FFFFFFFu;   // |w| from the high word of w

struct TcArgs {
    const unsigned short* V;  // f16 codes, column c at V + c * ld
    long long ld;
    int ncols;                // <= 128
    const double* W;          // n x k, column-major, leading dimension ldw
    long long ldw;
    long long n;
    int k;                    // <= 8
    float2* part;             // [gridDim.x][4][8][128]: double-float sums (see k_reduce_tc)
    int* eref;                // [gridDim.x][8]: their scale exponents
    int* fault;               // a wait timed out
    int* bad;                 // an input outside the exact range (|v| > 1, non-finite w)
};

// Operand tiles are K-major with the 128-byte swizzle: row m (one 128-byte line of 64 K
// values) at m * 128, its 16-byte chunk c stored at chunk position c ^ (m & 7), so eight
// consecutive rows spread one K chunk over all banks (for the stores here and for the
// tensor core's reads).  Tile bases are 1024-byte aligned; a K step of 16 values
// advances the start address by 32 bytes inside the swizzle atom.
__device__ __forceinline__ int swz(int m, int chunk) { return m * ROWB + ((chunk ^ (m & 7)) << 4); }

__device__ __forceinline__ uint64_t smem_desc(uint32_t addr)
{
    uint64_t d = (uint64_t)((addr >> 4) & 0x3FFF);
    d |= (uint64_t)1 << 16;                     // leading offset: unused for swizzled K-major
    d |= (uint64_t)((SBO >> 4) & 0x3FFF) << 32;
    d |= (uint64_t)1 << 46;                     // descriptor version (sm_100 family)
    d |= (uint64_t)2 << 61;                     // 128-byte swizzle
    return d;
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

// 16 consecutive TMEM columns of this warp's 32 lanes (completed by tmem_wait_ld)
__device__ __forceinline__ void tmem_ld16(uint32_t addr, uint32_t* r)
{
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(addr));
}

__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// Bounded wait that also gives up when another warp has recorded a timeout; the warp
// agrees on the outcome, so no lane is left at a warp-wide operation.
__device__ __forceinline__ bool warp_wait_or_abort(uint64_t* bar, unsigned parity, volatile int* abort_flag)
{
    bool ok = mbar_try_wait(bar, parity);
    if (!ok) {
        const long long t0 = clock64();
        while (!(ok = mbar_try_wait(bar, parity))) {
            if (*abort_flag) break;
            if (clock64() - t0 > WAIT_LIMIT_CYCLES) {
                *abort_flag = 1;
                break;
            }
        }
    }
    return __all_sync(0xffffffffu, ok);
}

__device__ __forceinline__ __half2 h2bits(unsigned int u) { return *reinterpret_cast<const __half2*>(&u); }
__device__ __forceinline__ unsigned int bits2(__half2 h) { return *reinterpret_cast<const unsigned int*>(&h); }
__device__ __forceinline__ float pow2f(int e) { return e < -126 ? 0.f : __int_as_float((127 + e) << 23); }

// Cut 8 codes (rows 8g .. 8g+7 of one column) into the digit planes at dst (hi) and
// dst + A_PLANE (lo); vover stays zero while every |v| <= 1.  Every step is exact in FP16 for |v| <= 1: the magic-number
// roundings t = fma(x, 2^j, 1536) keep |x 2^j| <= 256, so t lies in [1024, 2048) where
// the FP16 spacing is 1; the remainders are multiples of the code's spacing small enough
// to be representable (FP16 subnormals are kept).
__device__ __forceinline__ void cut_v(uint4 raw, unsigned char* dst, __half2& vover)
{
    const __half2 c4 = h2bits(0x44004400u), magic = h2bits(0x66006600u), cmq = h2bits(0xB400B400u);
    const __half2 c2048 = h2bits(0x68006800u), c512 = h2bits(0x60006000u), cm2m11 = h2bits(0x90009000u);
    const __half2 c4096 = h2bits(0x6C006C00u);
    const unsigned int w[4] = {raw.x, raw.y, raw.z, raw.w};
    unsigned int oh[4], ol[4];
#pragma unroll
    for (int i = 0; i < 4; i++) {
        const __half2 v = h2bits(w[i]);
        vover = __hadd2(vover, __hfma2_relu(v, v, h2bits(0xBC00BC00u)));   // += max(v^2 - 1, 0)
        const __half2 c = __hsub2(__hfma2(v, c4, magic), magic);          // rint(4 v)
        const __half2 r = __hfma2(c, cmq, v);                             // v - c/4, |r| <= 1/8
        const __half2 f = __hsub2(__hfma2(r, c2048, magic), magic);       // rint(2048 r)
        oh[i] = bits2(__hfma2(c, c512, f));                               // hi = rint(2048 v)
        ol[i] = bits2(__hmul2(__hfma2(f, cm2m11, r), c4096));             // lo = 2^12 (v - hi/2048)
    }
    *reinterpret_cast<uint4*>(dst) = make_uint4(oh[0], oh[1], oh[2], oh[3]);
    *reinterpret_cast<uint4*>(dst + A_PLANE) = make_uint4(ol[0], ol[1], ol[2], ol[3]);
}

// y = trunc(w 2^(54 - E)) from the bits of w (|w| < 2^E, so the shift below is >= -1);
// zero and subnormal w (below 2^-1022) contribute nothing.  Branch-free.
__device__ __forceinline__ long long w_scaled(unsigned long long u, int E)
{
    const int ex = (int)((u >> 52) & 0x7FF);
    const unsigned long long m = (u & 0xFFFFFFFFFFFFFull) | (1ull << 52);
    const int sh = E + (1023 - 2) - ex;     // y = m 2^(ex - 1075 + 54 - E) = m 2^-sh
    unsigned long long q = sh < 0 ? m << 1 : m >> (sh > 63 ? 63 : sh);
    q = (ex == 0 || sh > 63 || E <= E_ZERO || E >= E_BAD) ? 0ull : q;
    return (u >> 63) ? -(long long)q : (long long)q;
}

// (S, C) += x per component (TwoSum; x exact)
__device__ __forceinline__ void df2_add(float2& S, float2& C, float2 x)
{
    const float2 m1 = f2_neg1();
    const float2 s = __fadd2_rn(S, x);
    const float2 bb = __ffma2_rn(S, m1, s);          // s - S
    const float2 t1 = __ffma2_rn(bb, m1, s);         // s - bb
    const float2 t2 = __ffma2_rn(t1, m1, S);         // S - (s - bb)
    const float2 u = __ffma2_rn(bb, m1, x);          // x - bb
    C = __fadd2_rn(C, __fadd2_rn(t2, u));
    S = s;
}

// add TMEM columns N0 .. N0+CNT-1 of one slice (column n = 8 b + r', vector r = r' xor
// (b >= 8 ? 4 : 0)) times 2^(4 b) to the per-vector-pair double-float sums
template <int N0, int CNT>
__device__ __forceinline__ void drain_cols(const uint32_t* v, float2* S, float2* C)
{
#pragma unroll
    for (int i = 0; i < CNT; i += 2) {
        const int n = N0 + i, b = n >> 3, pr = ((n & 7) >> 1) ^ (b >= 8 ? 2 : 0);
        const float sc = __int_as_float((127 + 4 * b) << 23);
        df2_add(S[pr], C[pr], __fmul2_rn(make_float2(__uint_as_float(v[i]), __uint_as_float(v[i + 1])),
                                         make_float2(sc, sc)));
    }
}

// E with max |w| < 2^E from the largest high word of |w| in a block (the exponent field
// decides; blocks of zeros and subnormals contribute nothing)
__device__ __forceinline__ int block_exponent(unsigned int mb)
{
    if (mb < 0x00100000u) return E_ZERO;
    if (mb >= 0x7FF00000u) return E_BAD;
    return (int)(mb >> 20) - 1022;
}

struct Feed {              // one producer thread's inputs of a chunk
    uint4 v0, v1;          // two 8-code groups of its basis column
    unsigned long long w;  // the bits of one entry of W
};

__global__ void __launch_bounds__(TC_THREADS, 1) k_dot_multi_tc(TcArgs a)
{
    extern __shared__ unsigned char tc_raw[];
    unsigned char* sm = reinterpret_cast<unsigned char*>(((size_t)tc_raw + 1023) & ~(size_t)1023);
    // ebar[b & 1]: the producers' maxima of block b are written; eready: E of the next
    // block is published (one phase per block)
    __shared__ __align__(8) uint64_t full[NBUF], empty[NBUF], tfull[2], tempty[2], ebar[2], eready;
    __shared__ uint32_t tbase;
    __shared__ int abort_flag, bad_flag;
    __shared__ unsigned int wmax[2][PRODUCERS][4];   // per block parity and warp: maxima of its 4 vectors
    __shared__ int eslot[4][NVEC], erun[4][NVEC];       // per block (mod 4): E_p and Eref_p
    // running double-float sums: [slice * 2 + digit half][pair of vectors][column]
    __shared__ float2 accS[4][4][TC_M], accC[4][4][TC_M];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const long long nch = (a.n + KC - 1) / KC;                     // chunks of the whole product
    const long long c0 = (long long)blockIdx.x * nch / gridDim.x;  // this CTA's chunks
    const int nq = (int)(((long long)blockIdx.x + 1) * nch / gridDim.x - c0);
    const long long pfirst = c0 / CPB;                             // block of the first chunk
    const long long rbeg = c0 * KC, rend = min(a.n, (c0 + nq) * KC); // this CTA's rows

    // zero the chunk buffers once: padding columns and vectors beyond k stay zero
    for (int i = tid; i < NBUF * BUF / 16; i += TC_THREADS) reinterpret_cast<uint4*>(sm)[i] = make_uint4(0, 0, 0, 0);
    for (int i = tid; i < 4 * 4 * TC_M; i += TC_THREADS) {
        (&accS[0][0][0])[i] = make_float2(0.f, 0.f);
        (&accC[0][0][0])[i] = make_float2(0.f, 0.f);
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(&tbase)),
                     "r"(TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        abort_flag = 0;
        bad_flag = 0;
        for (int b = 0; b < NBUF; b++) {
            mbar_init(&full[b], PRODUCERS);
            mbar_init(&empty[b], 1);
        }
        for (int b = 0; b < 2; b++) {
            mbar_init(&tfull[b], 1);
            mbar_init(&tempty[b], PRODUCERS);
        }
        mbar_init(&ebar[0], PRODUCERS);
        mbar_init(&ebar[1], PRODUCERS);
        mbar_init(&eready, 1);
        mbar_init_fence();
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tbase;
    const uint32_t sbase = smem_addr(sm);
    volatile int* abort_v = &abort_flag;

    if (warp == MMA_WARP) {
        const uint32_t idesc = (1u << 4) | ((uint32_t)(TC_N >> 3) << 17) | ((uint32_t)(TC_M >> 4) << 24);
        int buf = 0, use = 0;           // chunk buffer and how often it has been filled before
        unsigned cnt[NBUF] = {0u, 0u, 0u};
        const int plast = (int)((c0 + nq - 1) / CPB - pfirst);
        // E of block b (lanes 0-7: vector r = lane) from the producers' maxima, published
        // on eready; by the time this runs the maxima are written (see below)
        auto exponents = [&](int b) -> bool {
            if (!warp_wait_or_abort(&ebar[b & 1], (b >> 1) & 1, abort_v)) return false;
            if (lane < NVEC) {
                unsigned int M = 0;
#pragma unroll
                for (int i = 0; i < 8; i++) M = max(M, wmax[b & 1][(lane >> 2) + 2 * i][lane & 3]);
                const int E = block_exponent(M);
                const int prev = b > 0 ? erun[(b - 1) & 3][lane] : E_ZERO;
                eslot[b & 3][lane] = E;
                erun[b & 3][lane] = (E == E_BAD || E == E_ZERO) ? prev : max(prev, E);
                if (E == E_BAD) atomicOr(&bad_flag, 1);
            }
            __syncwarp();
            if (lane == 0) mbar_arrive(&eready);
            return true;
        };
        int enext = 1;                  // next block whose exponents are due
        bool ok = nq > 0 ? exponents(0) : true;
        for (int q = 0; ok && q < nq; q++) {
            if (!warp_wait_or_abort(&full[buf], use & 1, abort_v)) break;
            const long long gq = c0 + q;
            const int jpos = (int)(gq % CPB), pi = (int)(gq / CPB - pfirst), set = pi & 1;
            const bool first = q == 0 || jpos == 0, last = q == nq - 1 || jpos == CPB - 1;
            // E of block pi + 1: its maxima were written by every producer at the start of
            // block pi (before their arrival on this chunk's buffer); published two chunks
            // into block pi, or at its last chunk, well before block pi + 1 needs it
            const int qstart = pi == 0 ? 0 : (int)((pfirst + pi) * CPB - c0);
            if (enext == pi + 1 && enext <= plast && (q - qstart >= 2 || last)) {
                if (!exponents(enext)) break;
                enext++;
            }
            // the sums of block pi - 2 (same tensor memory) must have been read
            if (first && pi >= 2 && !warp_wait_or_abort(&tempty[set], ((pi - 2) >> 1) & 1, abort_v)) break;
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            if (lane == 0) {
                const uint32_t ab = sbase + buf * BUF, bb = ab + SV * A_PLANE;
#pragma unroll
                for (int s = 0; s < SV; s++) {
#pragma unroll
                    for (int kk = 0; kk < KC / 16; kk++)
                        mma_f16(tmem + (uint32_t)(set * SET_COLS + s * SLICE_COLS),
                                smem_desc(ab + s * A_PLANE + kk * 32), smem_desc(bb + kk * 32), idesc,
                                (first && kk == 0) ? 0 : 1);
                }
                mma_commit(&empty[buf]);
                if (last) mma_commit(&tfull[set]);
            }
            __syncwarp();
#pragma unroll
            for (int b = 0; b < NBUF; b++) cnt[b] += (b == buf);
            if (++buf == NBUF) { buf = 0; use++; }
        }
        // no MMA may still run when tensor memory is freed (bounded waits)
#pragma unroll
        for (int b = 0; b < NBUF; b++)
            if (cnt[b] > 0) warp_wait(&empty[b], (cnt[b] - 1) & 1);
    } else {
        // V role: warp w cuts basis columns 8w .. 8w+7; lane = column (lane & 7) and 8-row
        // groups (K chunks) (lane >> 3) and (lane >> 3) + 4, so 8 lanes store one chunk of 8
        // consecutive rows: all banks.  Columns beyond ncols are cut from zeros, so all
        // warps do the same work.
        const int vc = warp * 8 + (lane & 7);
        const bool vlive = vc < a.ncols;
        const unsigned short* vcol = a.V + (long long)(vlive ? vc : 0) * a.ld + (lane >> 3) * 8;
        const int voff = swz(vc, lane >> 3), voff2 = swz(vc, (lane >> 3) + 4);
        // W role: vector r, row 8g + 2jj + p of the chunk; lanes p = 0 / 1 hold rows 2j / 2j+1,
        // exchange words and write digits 0-7 / 8-15 of both rows (digits 14 and 15 land in
        // the unused rows 112-127 of the plane; vectors beyond k write zero digits).  Digit
        // d of the lane's half is operand row n = 8 (8p + d) + (r ^ 4p): a warp's store
        // covers 8 distinct (n & 7) x 4 word positions, all banks.
        const int p = lane & 1, jj = (lane >> 1) & 3, r = (lane >> 3) + 4 * (warp & 1), g = warp >> 1;
        const int wrow = 8 * g + 2 * jj + p;
        const bool wlive = r < a.k;
        const double* wcol = a.W + (long long)(wlive ? r : 0) * a.ldw;
        const int woff = SV * A_PLANE + swz(64 * p + (r ^ (4 * p)), g) + jj * 4;
        // drain role: TMEM lane quadrant, V slice and digit half (digits 0-7 / 8-13)
        const int quad = warp & 3, dsl = (warp >> 2) & 1, dh = warp >> 3;
        const int col = quad * 32 + lane, h = dsl * 2 + dh;
        __half2 vover = h2bits(0u);

        auto load = [&](int q, Feed& F) {
            const long long r0 = (c0 + q) * KC;
            F.v0 = vlive ? __ldcs(reinterpret_cast<const uint4*>(vcol + r0)) : make_uint4(0, 0, 0, 0);
            F.v1 = vlive ? __ldcs(reinterpret_cast<const uint4*>(vcol + r0 + 32)) : make_uint4(0, 0, 0, 0);
            F.w = (wlive && r0 + wrow < a.n) ? __ldcs(reinterpret_cast<const unsigned long long*>(wcol) + r0 + wrow) : 0ull;
        };
        // high word of this thread's row of chunk j of block blk, 0 outside this CTA's rows
        // (the sign is masked off where the value is used, so the load stays in flight)
        auto wbits = [&](long long blk, int j) -> unsigned int {
            const long long row = blk * KB + (long long)j * KC + wrow;
            return (wlive && row >= rbeg && row < rend) ? __ldg(reinterpret_cast<const unsigned int*>(wcol + row) + 1)
                                                         : 0u;
        };
        // this warp's maxima of block b (per vector) for the MMA warp, which publishes E
        auto contribute = [&](int b, unsigned int mb) {
#pragma unroll
            for (int o = 1; o < 8; o <<= 1) mb = max(mb, __shfl_xor_sync(0xffffffffu, mb, o));
            if ((lane & 7) == 0) wmax[b & 1][warp][lane >> 3] = mb;
            __syncwarp();
            if (lane == 0) mbar_arrive(&ebar[b & 1]);
        };

        // the sums of block d: read this warp's TMEM quadrant of its slice and digit half,
        // release the set, and add them (scaled) to the running double-float sums
        auto drain = [&](int d) -> bool {
            const int set = d & 1;
            if (!warp_wait_or_abort(&tfull[set], (d >> 1) & 1, abort_v)) return false;
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t taddr =
                tmem + ((uint32_t)(quad * 32) << 16) + (uint32_t)(set * SET_COLS + dsl * SLICE_COLS);
            float2 S[4], C[4];
#pragma unroll
            for (int i = 0; i < 4; i++) { S[i] = make_float2(0.f, 0.f); C[i] = make_float2(0.f, 0.f); }
            uint32_t v[16];
            if (dh == 0) {
                tmem_ld16(taddr, v);
                tmem_wait_ld();
                drain_cols<0, 16>(v, S, C);
                tmem_ld16(taddr + 16, v);
                tmem_wait_ld();
                drain_cols<16, 16>(v, S, C);
                tmem_ld16(taddr + 32, v);
                tmem_wait_ld();
                drain_cols<32, 16>(v, S, C);
                tmem_ld16(taddr + 48, v);
                tmem_wait_ld();
            } else {
                tmem_ld16(taddr + 64, v);
                tmem_wait_ld();
                drain_cols<64, 16>(v, S, C);
                tmem_ld16(taddr + 80, v);
                tmem_wait_ld();
                drain_cols<80, 16>(v, S, C);
                tmem_ld16(taddr + 96, v);
                tmem_wait_ld();
            }
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            __syncwarp();
            if (lane == 0) mbar_arrive(&tempty[set]);
            if (dh == 0) drain_cols<48, 16>(v, S, C);
            else drain_cols<96, 16>(v, S, C);
            // this block x 2^(E_d - Eref_d), the running sums x 2^(Eref_{d-1} - Eref_d)
#pragma unroll
            for (int pr = 0; pr < 4; pr++) {
                float ks[2], kr[2];
#pragma unroll
                for (int e = 0; e < 2; e++) {
                    const int rr = 2 * pr + e, Ed = eslot[d & 3][rr], Er = erun[d & 3][rr];
                    const int Ep = d > 0 ? erun[(d - 1) & 3][rr] : E_ZERO;
                    ks[e] = (Ed == E_ZERO || Ed == E_BAD || Ed - Er < -DROP) ? 0.f : pow2f(Ed - Er);
                    kr[e] = (Ep == E_ZERO || Ep - Er < -DROP) ? 0.f : pow2f(Ep - Er);
                }
                const float2 kS = make_float2(ks[0], ks[1]), kR = make_float2(kr[0], kr[1]);
                float2 As = __fmul2_rn(accS[h][pr][col], kR), Ac = __fmul2_rn(accC[h][pr][col], kR);
                df2_add(As, Ac, __fmul2_rn(S[pr], kS));
                Ac = __fadd2_rn(Ac, __fmul2_rn(C[pr], kS));
                const float2 s2 = __fadd2_rn(As, Ac);                       // renormalise
                accC[h][pr][col] = __ffma2_rn(__ffma2_rn(As, f2_neg1(), s2), f2_neg1(), Ac);
                accS[h][pr][col] = s2;
            }
            return true;
        };

        // maxima of the first two blocks (this CTA's rows of them) and the rows of the
        // third block that precede j0 (only the first block starts late); afterwards the
        // maxima of block p + 2 are gathered, one row per chunk, during block p
        const int j0 = (int)(c0 % CPB);
        const int plast = (int)((c0 + nq - 1) / CPB - pfirst);   // this CTA's last block index
        unsigned int nmax = 0;
        if (nq > 0) {
            unsigned int m = 0;
            for (int j = j0; j < CPB; j++) m = max(m, wbits(pfirst, j) & ABS_HI);
            contribute(0, m);
            if (plast >= 1) {
                m = 0;
                for (int j = 0; j < CPB; j++) m = max(m, wbits(pfirst + 1, j) & ABS_HI);
                contribute(1, m);
            }
            if (plast >= 2)
                for (int j = 0; j < j0; j++) nmax = max(nmax, wbits(pfirst + 2, j) & ABS_HI);
        }
        int Ecur = E_ZERO;
        if (nq > 0 && warp_wait_or_abort(&eready, 0, abort_v)) Ecur = eslot[0][r];
        unsigned int npend = 0;              // high word of one row of block p + 2, loaded a chunk ago
        int drained = 0, buf = 0, use = 0;
        int jpos = j0, pi = 0;               // position of the current chunk: block, chunk in block

        auto step = [&](int q, Feed& F) -> bool {
            if (q > 0 && jpos == 0) {        // block pi starts: hand over the maxima of pi + 1
                nmax = max(nmax, npend & ABS_HI);
                npend = 0;
                if (pi + 1 <= plast) contribute(pi + 1, nmax);
                nmax = 0;
                if (!warp_wait_or_abort(&eready, pi & 1, abort_v)) return false;
                Ecur = eslot[pi & 3][r];
            }
            // the MMAs that last read this buffer (NBUF chunks ago) must be complete
            if (use > 0 && !warp_wait_or_abort(&empty[buf], (use - 1) & 1, abort_v)) return false;
            unsigned char* B = sm + buf * BUF;
            const long long y = w_scaled(F.w, Ecur);
            cut_v(F.v0, B + voff, vover);
            cut_v(F.v1, B + voff2, vover);
            load(q + 2 < nq ? q + 2 : nq - 1, F);   // registers of chunk q are consumed
            const unsigned long long z = (unsigned long long)y + WBIAS;   // nibbles = digits + 8
            const unsigned int lo = (unsigned int)z, hi = (unsigned int)(z >> 32);
            const unsigned int other = __shfl_xor_sync(0xffffffffu, p ? lo : hi, 1);
            const unsigned int wa = p ? other : lo, wb = p ? hi : other;   // words of rows 2j, 2j+1
            // low nibble n: half(1024 + n) - 1032 = n - 8; high nibble n: half(1024 + 16 n) / 16 - 72
            const __half2 off = h2bits(0x64086408u), sixteenth = h2bits(0x2C002C00u), m72 = h2bits(0xD480D480u);
#pragma unroll
            for (int i = 0; i < 4; i++) {
                const unsigned int u = __byte_perm(wa, wb, i | (i << 4) | ((4 + i) << 8) | ((4 + i) << 12));
                const unsigned int ev = (u & 0x000F000Fu) | 0x64006400u, od = (u & 0x00F000F0u) | 0x64006400u;
                *reinterpret_cast<unsigned int*>(B + woff + 2 * i * SBO) = bits2(__hsub2(h2bits(ev), off));
                *reinterpret_cast<unsigned int*>(B + woff + (2 * i + 1) * SBO) = bits2(__hfma2(h2bits(od), sixteenth, m72));
            }
            nmax = max(nmax, npend & ABS_HI);
            npend = pi + 2 <= plast ? wbits(pfirst + pi + 2, jpos) : 0u;
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");   // visible to the tensor core
            __syncwarp();
            if (lane == 0) mbar_arrive(&full[buf]);
            if (++buf == NBUF) { buf = 0; use++; }
            // the previous block's sums, once this block is under way
            if (jpos >= 1)
                while (drained < pi)
                    if (!drain(drained++)) return false;
            if (++jpos == CPB) { jpos = 0; pi++; }
            return true;
        };

        Feed A{}, Bf{};
        if (nq > 0) load(0, A);
        if (nq > 1) load(1, Bf);
        for (int q = 0; !*abort_v && q < nq; q += 2) {
            if (!step(q, A)) break;
            if (q + 1 < nq && !step(q + 1, Bf)) break;
        }
        while (!*abort_v && nq > 0 && drained <= plast)
            if (!drain(drained++)) break;
        if (bits2(vover) & 0x7FFF7FFFu) atomicOr(&bad_flag, 1);   // some |v| > 1 (or not finite)
        // this CTA's double-float sums and their scale exponents
#pragma unroll
        for (int pr = 0; pr < 4; pr++) {
            a.part[(((long long)blockIdx.x * 4 + h) * 8 + pr * 2 + 0) * TC_M + col] = accS[h][pr][col];
            a.part[(((long long)blockIdx.x * 4 + h) * 8 + pr * 2 + 1) * TC_M + col] = accC[h][pr][col];
        }
        if (warp == 0 && lane < NVEC) a.eref[blockIdx.x * NVEC + lane] = nq > 0 ? erun[plast & 3][lane] : E_ZERO;
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS) : "memory");
    if (tid == 0) {
        if (bad_flag) atomicOr(a.bad, 1);
        if (abort_flag && a.fault) atomicExch(a.fault, 1);
    }
}

// H[c][r] = scales[c] * sum over CTAs (in CTA order) and the four (slice, digit half)
// sums of (S + C) 2^(Eref - 54 + ps): one warp per entry, so the FP64 work (slow on this
// GPU) is spread over the device
__global__ void k_reduce_tc(const float2* part, const int* eref, int nparts, int ncols, int k, int ldh,
                            const double* scales, const int* bad, const int* fault, double* H)
{
    const int i = (int)(((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5), lane = threadIdx.x & 31;
    if (i >= ncols * k) return;
    const int col = i / k, r = i - col * k, pr = r >> 1, e = r & 1;
    double sum = 0.0;
    for (int t = lane; t < nparts * 4; t += 32) {
        const int b = t >> 2, h = t & 3, ps = (h >> 1) == 0 ? -11 : -12;   // slice hi / lo
        const int E = eref[b * NVEC + r];
        if (E <= E_ZERO || E >= E_BAD) continue;
        const float2 S = part[(((long long)b * 4 + h) * 8 + pr * 2 + 0) * TC_M + col];
        const float2 C = part[(((long long)b * 4 + h) * 8 + pr * 2 + 1) * TC_M + col];
        const int x = E - WSHIFT + ps;
        const double sc = x < -1022 ? 0.0 : __longlong_as_double((long long)(x + 1023) << 52);
        sum = __fma_rn(e ? df_to_double(S.y, C.y) : df_to_double(S.x, C.x), sc, sum);
    }
    sum = warp_sum(sum);
    if (lane == 0)
        H[(long long)col * ldh + r] = (*bad || *fault) ? __longlong_as_double(0x7FF8000000000000ll) : sum * scales[col];
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
// layout: [unused, fault, bad | partials | exponents].
size_t cbg_tc_multi_workspace(int64_t ld)
{
    (void)ld;
    const size_t g = (size_t)tc_grid();
    return 256 + g * 4 * 8 * TC_M * sizeof(float2) + g * NVEC * sizeof(int);
}

int cbg_tc_multi(int64_t n, int ncols, const void* V, int64_t ld, const double* scales, int k, int ldh, const double* W,
                 int64_t ldw, double* H, void* workspace, cudaStream_t s, int** fault_out)
{
    unsigned char* ws = static_cast<unsigned char*>(workspace);
    int* fault = reinterpret_cast<int*>(ws + 4);
    int* bad = reinterpret_cast<int*>(ws + 8);
    const int grid = tc_grid();
    float2* part = reinterpret_cast<float2*>(ws + 256);
    int* eref = reinterpret_cast<int*>(ws + 256 + (size_t)grid * 4 * 8 * TC_M * sizeof(float2));
    if (fault_out) *fault_out = fault;
    if (cudaMemsetAsync(ws, 0, 16, s) != cudaSuccess) return CBG_ERR_CUDA;
    static const bool attr = [] {
        cudaFuncSetAttribute(k_dot_multi_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, TC_SMEM);
        return true;
    }();
    (void)attr;
    TcArgs a{};
    a.V = static_cast<const unsigned short*>(V);
    a.ld = ld;
    a.ncols = ncols;
    a.W = W;
    a.ldw = ldw;
    a.n = n;
    a.k = k;
    a.part = part;
    a.eref = eref;
    a.fault = fault;
    a.bad = bad;
    k_dot_multi_tc<<<grid, TC_THREADS, TC_SMEM, s>>>(a);
    k_reduce_tc<<<(ncols * k * 32 + 255) / 256, 256, 0, s>>>(part, eref, grid, ncols, k, ldh, scales, bad, fault, H);
    return cudaGetLastError() == cudaSuccess ? CBG_OK : CBG_ERR_CUDA;
}
