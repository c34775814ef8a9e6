// mlp_tc.cu -- the learned preconditioner's per-row network on the 5th-generation tensor
// cores: forward pass, backward pass, and one fused training pass (forward, loss from the
// per-row pair statistics, backward, weight gradients).
//
// Precision contract: every tensor-core operand is BF16 and every product sum accumulates
// in FP32 in tensor memory (the weight gradients over all of a CTA's rows).  The inputs
// of layers 1 and 2 (features, H1) and the output gradient enter as split pairs
// hi + lo of BF16 values (about 16 significant bits; the lo half is a second K block
// against a copy of the same weights), so the ReLU decisions are taken on FP32-accurate
// pre-activations; H2 and the backward's dZ2, dZ1 and the gradient products' operands
// are single BF16 values.  Biases, ReLU, the loss and its gradient are FP32 on the CUDA
// cores; the cross-CTA gradient sum is FP64 (k_grad_reduce).
//
// One CTA per SM, 128 threads: thread t owns row t of a 128-row tile and tensor-memory
// lane t (warp w reads lanes 32w .. 32w+31).  Per tile, with D = A B^T and every operand a
// K-major, 128-byte-swizzled tile in shared memory (cbg_tc.cuh):
//   layer 1  Z1 = F  W1^T       M 128, N 64, K 16 (7 features hi, 7 lo, zero padded)
//   layer 2  Z2 = H1 W2^T       M 128, N 64, K 2 x 64    H1 = relu(Z1 + b1), hi and lo
//   layer 3  Y  = H2 W3^T       M 128, N 16, K 64        H2 = relu(Z2 + b2), out = Y + b3
//   dH2 = Gout W3               M 128, N 64, K 16        Gout = dL/dout, hi and lo
//   dH1 = dZ2 W2                M 128, N 64, K 64        dZ2 = dH2 * [Z2 + b2 > 0]
//   [gW2 | gb2 ; gW1 | gb1] += [dZ2^T ; dZ1^T] [H1^T ; F^T ; 1]^T     M 128, N 80, K = rows
//   gW3^T += [H2^T ; H1^T] [Gout^T]^T                                  M 128, N 16, K = rows
// (dZ1 = dH1 * [Z1 + b1 > 0]; the transposed activations are written by the epilogues
// next to the row-major copies; the ones row turns the bias gradients into extra output
// columns; rows below H1^T in the second product only fill M and are not read).  The
// weight-gradient sums stay in tensor memory across the CTA's tiles and are written once.
// The tile's inputs are staged with cp.async one phase ahead (features after layer 1 of
// the previous tile, statistics after its loss).  Every wait on the tensor core is
// bounded: a wait that runs out sets *fault and the CTA leaves the tile loop.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>

#include "cbg_device.cuh"
#include "cbg_mlp.h"
#include "cbg_tc.cuh"

namespace cbg {
namespace {

constexpr int MT = 128;                        // threads: one per row of a tile
constexpr int ROWS = MLP_ROWS;
constexpr int TM_COLS = 256;                   // tensor-memory columns of a CTA
constexpr int C_Z1 = 0, C_Z2 = 64, C_Y = 128, C_G = 144, C_G3 = 224;
constexpr int NG = 80;                         // [H1^T ; F^T ; 1 ; 0]: 64 + 7 + 1 + 8 rows
constexpr int ONES_ROW = 64 + NH + NIN;        // row 135 of the X block
// shared memory, bytes from the 1024-aligned base
constexpr int S_W1 = 0;                        // [64 o][K: W1 row, copy at K 8] B of layer 1
constexpr int S_W2 = S_W1 + 64 * TC_ROWB;      // [64 o][64 q]                 B of layer 2
constexpr int S_W2T = S_W2 + 64 * TC_ROWB;     // [64 q][64 o]                 B of dH1
constexpr int S_W3T = S_W2T + 64 * TC_ROWB;    // [64 o][K: W3 col, copy at K 8] B of dH2
constexpr int S_W3 = S_W3T + 64 * TC_ROWB;     // [16 k][64 o] (rows 7-15 zero) B of layer 3
constexpr int S_FG = S_W3 + 16 * TC_ROWB;      // [128 r][F hi, lo: K 0-15 | Gout hi, lo: K 16-31]
constexpr int S_H1 = S_FG + ROWS * TC_ROWB;    // [128 r][64] H1 hi            A of layer 2
constexpr int S_H1L = S_H1 + ROWS * TC_ROWB;   // [128 r][64] H1 lo            A of layer 2 (second K block)
constexpr int S_H2 = S_H1L + ROWS * TC_ROWB;   // [128 r][64]                  A of layer 3
constexpr int S_D2 = S_H2 + ROWS * TC_ROWB;    // [128 r][64]                  A of dH1
constexpr int X_BYTES = 144 * TC_ROWB;         // per 64-row K tile: [H2^T | H1^T | F^T, 1, 0]
constexpr int S_X = S_D2 + ROWS * TC_ROWB;
constexpr int Y_BYTES = 128 * TC_ROWB;         // per K tile: [dZ2^T | dZ1^T]
constexpr int S_Y = S_X + 2 * X_BYTES;
constexpr int Z_BYTES = 16 * TC_ROWB;          // per K tile: [Gout^T | 0]
constexpr int S_Z = S_Y + 2 * Y_BYTES;
constexpr int S_OPS_END = S_Z + 2 * Z_BYTES;   // end of the tensor-core operands
// staged inputs of a tile (cp.async) and the biases
constexpr int S_FEAT = S_OPS_END;              // 128 x 7 floats
constexpr int S_GOUT = S_FEAT + ROWS * 28;     // 128 x 7 floats (MLP_BWD)
constexpr int S_G = S_GOUT + ROWS * 28;        // 128 x 49 floats (MLP_TRAIN)
constexpr int S_C = S_G + ROWS * 196;          // 128 x 7 floats
constexpr int S_D = S_C + ROWS * 28;           // 128 floats
constexpr int S_DIAG = S_D + ROWS * 4;         // 128 doubles
constexpr int S_MASK = S_DIAG + ROWS * 8;      // 128 bytes
constexpr int S_BIAS = S_MASK + ROWS;          // b1[64], b2[64], b3[7] floats
constexpr int S_END = S_BIAS + (2 * NH + 8) * 4;
constexpr int MLP_SMEM = S_END + 1024;         // + alignment slack
static_assert(S_FG % 1024 == 0 && S_X % 1024 == 0 && S_Y % 1024 == 0 && S_Z % 1024 == 0 && X_BYTES % 1024 == 0,
              "operand tiles start on 1024-byte swizzle atoms");
static_assert(MLP_SMEM <= 232448, "fits the opt-in shared memory of one CTA");

__device__ __forceinline__ void cp_async16(void* dst, const void* src, int bytes)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(smem_addr(dst)), "l"(src), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N> __device__ __forceinline__ void cp_async_wait()
{
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// Stage `total` bytes of a tile's segment (16-byte aligned) into shared memory; bytes at
// or beyond `valid` (rows past n) read as zeros.
__device__ __forceinline__ void stage(unsigned char* dst, const void* src, int total, long long valid)
{
    const unsigned char* s = static_cast<const unsigned char*>(src);
    for (int j = threadIdx.x; j < total / 16; j += MT) {
        const long long v = valid - 16ll * j;
        const int bytes = v >= 16 ? 16 : (v > 0 ? (int)v : 0);
        cp_async16(dst + 16 * j, bytes > 0 ? s + 16 * j : s, bytes);
    }
}

__device__ __forceinline__ unsigned int bf2(float lo, float hi)
{
    const __nv_bfloat162 b = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<const unsigned int*>(&b);
}
__device__ __forceinline__ float bf_lo(unsigned int u) { return __uint_as_float(u << 16); }
__device__ __forceinline__ float bf_hi(unsigned int u) { return __uint_as_float(u & 0xFFFF0000u); }
// the rounding residuals of a packed pair: (x0, x1) - (hi pair), again as a BF16 pair
// (the differences are exact in FP32)
__device__ __forceinline__ unsigned int bf2_rest(float x0, float x1, unsigned int hi)
{
    return bf2(x0 - bf_lo(hi), x1 - bf_hi(hi));
}

// a BF16 value of parameter p (held in FP32) as the 16 bits of an operand element
__device__ __forceinline__ unsigned short pbits(const float* P, int idx)
{
    return (unsigned short)(__float_as_uint(P[idx]) >> 16);
}

// element (row m, K index k) of a K-major swizzled operand tile
__device__ __forceinline__ unsigned short* opnd(unsigned char* tile, int m, int k)
{
    return reinterpret_cast<unsigned short*>(tile + tc_swz(m, k >> 3) + (k & 7) * 2);
}

// Eight BF16 values of this thread's row (four packed pairs) into chunk `chunk` of a
// row-major operand row; put_col writes `cnt` values transposed instead: value o0 + i to
// row r0 + o0 + i of a K tile, at the K index of this thread's row (t mod 64)
__device__ __forceinline__ void put_row8(unsigned char* base, int row, int chunk, const unsigned int* pk)
{
    *reinterpret_cast<uint4*>(base + tc_swz(row, chunk)) = make_uint4(pk[0], pk[1], pk[2], pk[3]);
}
__device__ __forceinline__ void put_col(unsigned char* ktile, int r0, int o0, int cnt, int t, const unsigned int* pk)
{
    const int kc = (t & 63) >> 3, ke = (t & 7) * 2;
    for (int i = 0; i < cnt; i++) {
        const unsigned short h = (unsigned short)((i & 1) ? (pk[i >> 1] >> 16) : (pk[i >> 1] & 0xFFFFu));
        *reinterpret_cast<unsigned short*>(ktile + tc_swz(r0 + o0 + i, kc) + ke) = h;
    }
}

template <int MODE>
__global__ void __launch_bounds__(MT, 1) k_mlp_tc(MlpArgs a)
{
    extern __shared__ unsigned char mlp_raw[];
    unsigned char* sm = reinterpret_cast<unsigned char*>(((size_t)mlp_raw + 1023) & ~(size_t)1023);
    __shared__ __align__(8) uint64_t mbar;
    __shared__ uint32_t tbase;
    __shared__ float red_b3[MT / 32][8];
    __shared__ double red_l[MT / 32];
    const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
    const long long ntiles = (a.n + ROWS - 1) / ROWS;
    constexpr bool BACK = MODE != MLP_FWD;

    // operands: zero everything once (padding of K, unused rows), then the constant
    // rows (ones) and the weights in their five operand layouts
    for (int i = t; i < S_OPS_END / 16; i += MT) reinterpret_cast<uint4*>(sm)[i] = make_uint4(0u, 0u, 0u, 0u);
    if (warp == 0) tc_alloc(&tbase, TM_COLS);
    if (t == 0) {
        mbar_init(&mbar, 1);
        mbar_init_fence();
    }
    __syncthreads();
    const float* P = a.params;
    for (int i = t; i < NH * 64; i += MT) {              // W2 and its transpose
        const int o = i >> 6, q = i & 63;
        const unsigned short w = pbits(P, OFF_W2 + o * NH + q);
        *opnd(sm + S_W2, o, q) = w;
        *opnd(sm + S_W2T, q, o) = w;
    }
    for (int i = t; i < NH * NIN; i += MT) {             // W1, twice: against the hi and lo features
        const int o = i / NIN, k = i % NIN;
        const unsigned short w = pbits(P, OFF_W1 + o * NIN + k);
        *opnd(sm + S_W1, o, k) = w;
        *opnd(sm + S_W1, o, 8 + k) = w;
    }
    for (int i = t; i < NOUT * NH; i += MT) {            // W3, and its transpose twice (hi, lo Gout)
        const int k = i / NH, o = i % NH;
        const unsigned short w = pbits(P, OFF_W3 + k * NH + o);
        *opnd(sm + S_W3, k, o) = w;
        *opnd(sm + S_W3T, o, k) = w;
        *opnd(sm + S_W3T, o, 8 + k) = w;
    }
    float* sb = reinterpret_cast<float*>(sm + S_BIAS);
    for (int i = t; i < NH; i += MT) {
        sb[i] = P[OFF_B1 + i];
        sb[NH + i] = P[OFF_B2 + i];
    }
    if (t < NOUT) sb[2 * NH + t] = P[OFF_B3 + t];
    if (BACK)
        for (int i = t; i < 2 * 64; i += MT) {           // the ones row of both K tiles
            unsigned char* x = sm + S_X + (i >> 6) * X_BYTES;
            *opnd(x, ONES_ROW, i & 63) = 0x3F80;          // BF16 1.0
        }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tbase;
    const uint32_t tl = tmem + ((uint32_t)(warp * 32) << 16);   // this warp's lanes
    const uint32_t sbase = smem_addr(sm);
    const float* b1 = sb;
    const float* b2 = sb + NH;
    const float* b3 = sb + 2 * NH;

    auto issue_inputs = [&](long long tile) {
        const long long r0 = tile * ROWS, rows = a.n - r0 < ROWS ? a.n - r0 : ROWS;
        stage(sm + S_FEAT, a.feat + r0 * NIN, ROWS * 28, rows * 28);
        if (MODE == MLP_BWD) stage(sm + S_GOUT, a.gout + r0 * NOUT, ROWS * 28, rows * 28);
        cp_async_commit();
    };
    auto issue_stats = [&](long long tile) {
        const long long r0 = tile * ROWS, rows = a.n - r0 < ROWS ? a.n - r0 : ROWS;
        stage(sm + S_G, a.G + r0 * 49, ROWS * 196, rows * 196);
        stage(sm + S_C, a.c + r0 * 7, ROWS * 28, rows * 28);
        stage(sm + S_D, a.d + r0, ROWS * 4, rows * 4);
        stage(sm + S_DIAG, a.diag + r0, ROWS * 8, rows * 8);
        stage(sm + S_MASK, a.mask + r0, ROWS, rows);
        cp_async_commit();
    };
    unsigned phase = 0;
    bool ok = true;
    // all threads: the MMAs committed last have completed (bounded), agreed block-wide
    auto mma_wait = [&]() -> bool {
        const bool mine = mbar_wait(&mbar, phase & 1u);
        phase++;
        const bool all = __syncthreads_and(mine) != 0;
        tc_fence_after();
        return all;
    };
    // the operand stores of every thread are visible to the tensor core, and its
    // tensor-memory loads are complete, before thread 0 issues the next MMAs
    auto to_tensor_core = [&]() {
        tc_fence_proxy();
        tc_fence_before();
        __syncthreads();
    };
    auto mma = [&](int col, int a_off, int b_off, int N, int ksteps, int acc0) {
        const uint32_t id = tc_idesc(128, N, true);
        for (int kk = 0; kk < ksteps; kk++)
            tc_mma(tmem + (uint32_t)col, tc_desc(sbase + a_off + kk * 32), tc_desc(sbase + b_off + kk * 32), id,
                   (kk == 0 && !acc0) ? 0 : 1);
    };

    float gb3[NOUT];
#pragma unroll
    for (int k = 0; k < NOUT; k++) gb3[k] = 0.f;
    double loss = 0.0;
    bool first = true;
    const long long tile0 = blockIdx.x;
    if (tile0 < ntiles) {
        issue_inputs(tile0);
        if (MODE == MLP_TRAIN) issue_stats(tile0);
    }
    for (long long tile = tile0; ok && tile < ntiles; tile += gridDim.x) {
        const long long r0 = tile * ROWS, i = r0 + t;
        const bool valid = i < a.n;
        const int kt = t >> 6;                            // K tile of this row in the gradient products
        if (MODE == MLP_TRAIN) cp_async_wait<1>();
        else cp_async_wait<0>();
        __syncthreads();
        // ---- features: F (K 0-7 of the FG tile) and F^T (rows 128-134 of the X block)
        float gin[NOUT];
        {
            const float* f = reinterpret_cast<const float*>(sm + S_FEAT) + t * NIN;
            unsigned int pk[4] = {bf2(f[0], f[1]), bf2(f[2], f[3]), bf2(f[4], f[5]), bf2(f[6], 0.f)};
            unsigned int pl[4] = {bf2_rest(f[0], f[1], pk[0]), bf2_rest(f[2], f[3], pk[1]),
                                  bf2_rest(f[4], f[5], pk[2]), bf2_rest(f[6], 0.f, pk[3])};
            put_row8(sm + S_FG, t, 0, pk);
            put_row8(sm + S_FG, t, 1, pl);
            if (BACK) put_col(sm + S_X + kt * X_BYTES, 128, 0, NIN, t, pk);
            if (MODE == MLP_BWD) {
                const float* g = reinterpret_cast<const float*>(sm + S_GOUT) + t * NOUT;
#pragma unroll
                for (int k = 0; k < NOUT; k++) gin[k] = g[k];
            }
        }
        to_tensor_core();
        const long long next = tile + gridDim.x;
        if (next < ntiles) issue_inputs(next);            // the staging rows are consumed
        if (t == 0) {
            tc_fence_after();
            mma(C_Z1, S_FG, S_W1, 64, 1, 0);
            tc_commit(&mbar);
        }
        if (!(ok = mma_wait())) break;
        // ---- layer 1 epilogue: H1 = relu(Z1 + b1)
        unsigned long long m1 = 0ull, m2 = 0ull;
#pragma unroll
        for (int c0 = 0; c0 < NH; c0 += 16) {
            uint32_t v[16];
            tc_ld16(tl + C_Z1 + c0, v);
            tc_wait_ld();
            unsigned int pk[8], pl[8];
#pragma unroll
            for (int e = 0; e < 16; e += 2) {
                const float z0 = __uint_as_float(v[e]) + b1[c0 + e], z1 = __uint_as_float(v[e + 1]) + b1[c0 + e + 1];
                m1 |= (z0 > 0.f ? 1ull : 0ull) << (c0 + e);
                m1 |= (z1 > 0.f ? 1ull : 0ull) << (c0 + e + 1);
                const float h0 = fmaxf(z0, 0.f), h1 = fmaxf(z1, 0.f);
                pk[e >> 1] = bf2(h0, h1);
                pl[e >> 1] = bf2_rest(h0, h1, pk[e >> 1]);
            }
            put_row8(sm + S_H1, t, c0 >> 3, pk);
            put_row8(sm + S_H1, t, (c0 >> 3) + 1, pk + 4);
            put_row8(sm + S_H1L, t, c0 >> 3, pl);
            put_row8(sm + S_H1L, t, (c0 >> 3) + 1, pl + 4);
            if (BACK) put_col(sm + S_X + kt * X_BYTES, 64, c0, 16, t, pk);
        }
        to_tensor_core();
        if (t == 0) {
            tc_fence_after();
            mma(C_Z2, S_H1, S_W2, 64, 4, 0);
            mma(C_Z2, S_H1L, S_W2, 64, 4, 1);
            tc_commit(&mbar);
        }
        if (!(ok = mma_wait())) break;
        // ---- layer 2 epilogue: H2 = relu(Z2 + b2)
#pragma unroll
        for (int c0 = 0; c0 < NH; c0 += 16) {
            uint32_t v[16];
            tc_ld16(tl + C_Z2 + c0, v);
            tc_wait_ld();
            unsigned int pk[8];
#pragma unroll
            for (int e = 0; e < 16; e += 2) {
                const float z0 = __uint_as_float(v[e]) + b2[c0 + e], z1 = __uint_as_float(v[e + 1]) + b2[c0 + e + 1];
                m2 |= (z0 > 0.f ? 1ull : 0ull) << (c0 + e);
                m2 |= (z1 > 0.f ? 1ull : 0ull) << (c0 + e + 1);
                pk[e >> 1] = bf2(fmaxf(z0, 0.f), fmaxf(z1, 0.f));
            }
            put_row8(sm + S_H2, t, c0 >> 3, pk);
            put_row8(sm + S_H2, t, (c0 >> 3) + 1, pk + 4);
            if (BACK) put_col(sm + S_X + kt * X_BYTES, 0, c0, 16, t, pk);
        }
        to_tensor_core();
        if (t == 0) {
            tc_fence_after();
            mma(C_Y, S_H2, S_W3, 16, 4, 0);
            tc_commit(&mbar);
        }
        if (!(ok = mma_wait())) break;
        // ---- layer 3 epilogue: out = Y + b3
        float y[NOUT];
        {
            uint32_t v[16];
            tc_ld16(tl + C_Y, v);
            tc_wait_ld();
#pragma unroll
            for (int k = 0; k < NOUT; k++) y[k] = __uint_as_float(v[k]) + b3[k];
        }
        if (MODE == MLP_FWD) {
            if (valid) {
#pragma unroll
                for (int k = 0; k < NOUT; k++) a.out[i * NOUT + k] = y[k];
            }
            tc_fence_before();
            __syncthreads();                              // every row's loads done before the next tile's MMAs
            continue;
        }
        if (MODE == MLP_TRAIN) {
            // loss and dL/dout from the per-row statistics (quadratic in the seven P values)
            cp_async_wait<0>();
            __syncthreads();
            const float* G = reinterpret_cast<const float*>(sm + S_G) + t * 49;
            const float* cc = reinterpret_cast<const float*>(sm + S_C) + t * 7;
            const float dd = reinterpret_cast<const float*>(sm + S_D)[t];
            const double dg = reinterpret_cast<const double*>(sm + S_DIAG)[t];
            const unsigned int mk = sm[S_MASK + t];
            // 1 / a_ii in FP32 (an FP64 division per row would sit on GB300's narrow FP64 pipe
            // between two block barriers)
            const float id = valid ? __frcp_rn(f64_to_f32_rn(dg)) : 0.f;
            float p[7];
#pragma unroll
            for (int k = 0; k < 7; k++) p[k] = (mk >> k) & 1u ? y[k] * id : 0.f;
            float li = dd;
#pragma unroll
            for (int k = 0; k < 7; k++) {
                float gp = 0.f;
#pragma unroll
                for (int l = 0; l < 7; l++) gp = fmaf(G[k * 7 + l], p[l], gp);
                li = fmaf(p[k], gp - 2.f * cc[k], li);
                gin[k] = (mk >> k) & 1u ? 2.f * (gp - cc[k]) * id * (float)a.inv_npairs : 0.f;
            }
            if (valid) loss += (double)li;
            __syncthreads();                              // the statistics are consumed
            if (next < ntiles) issue_stats(next);
        }
        if (!valid) {
#pragma unroll
            for (int k = 0; k < NOUT; k++) gin[k] = 0.f;
        }
        // ---- Gout hi and lo (K 16-22 and 24-30 of the FG tile), Gout^T (rows 0-6 of the Z tile)
        {
            unsigned int pk[4] = {bf2(gin[0], gin[1]), bf2(gin[2], gin[3]), bf2(gin[4], gin[5]), bf2(gin[6], 0.f)};
            unsigned int pl[4] = {bf2_rest(gin[0], gin[1], pk[0]), bf2_rest(gin[2], gin[3], pk[1]),
                                  bf2_rest(gin[4], gin[5], pk[2]), bf2_rest(gin[6], 0.f, pk[3])};
            put_row8(sm + S_FG, t, 2, pk);
            put_row8(sm + S_FG, t, 3, pl);
            put_col(sm + S_Z + kt * Z_BYTES, 0, 0, NOUT, t, pk);
#pragma unroll
            for (int k = 0; k < NOUT; k++) gb3[k] += gin[k];
        }
        to_tensor_core();
        if (t == 0) {
            tc_fence_after();
            mma(C_Z2, S_FG + 32, S_W3T, 64, 1, 0);        // dH2 = Gout W3 (K 16-31: bytes 32..63)
            tc_commit(&mbar);
        }
        if (!(ok = mma_wait())) break;
        // ---- dZ2 = dH2 * relu'(layer 2): row-major (A of dH1) and transposed (Y rows 0-63)
#pragma unroll
        for (int c0 = 0; c0 < NH; c0 += 16) {
            uint32_t v[16];
            tc_ld16(tl + C_Z2 + c0, v);
            tc_wait_ld();
            unsigned int pk[8];
#pragma unroll
            for (int e = 0; e < 16; e += 2) {
                const float d0 = (m2 >> (c0 + e)) & 1ull ? __uint_as_float(v[e]) : 0.f;
                const float d1 = (m2 >> (c0 + e + 1)) & 1ull ? __uint_as_float(v[e + 1]) : 0.f;
                pk[e >> 1] = bf2(d0, d1);
            }
            put_row8(sm + S_D2, t, c0 >> 3, pk);
            put_row8(sm + S_D2, t, (c0 >> 3) + 1, pk + 4);
            put_col(sm + S_Y + kt * Y_BYTES, 0, c0, 16, t, pk);
        }
        to_tensor_core();
        if (t == 0) {
            tc_fence_after();
            mma(C_Z1, S_D2, S_W2T, 64, 4, 0);             // dH1 = dZ2 W2
            tc_commit(&mbar);
        }
        if (!(ok = mma_wait())) break;
        // ---- dZ1 = dH1 * relu'(layer 1): transposed (Y rows 64-127)
#pragma unroll
        for (int c0 = 0; c0 < NH; c0 += 16) {
            uint32_t v[16];
            tc_ld16(tl + C_Z1 + c0, v);
            tc_wait_ld();
            unsigned int pk[8];
#pragma unroll
            for (int e = 0; e < 16; e += 2) {
                const float d0 = (m1 >> (c0 + e)) & 1ull ? __uint_as_float(v[e]) : 0.f;
                const float d1 = (m1 >> (c0 + e + 1)) & 1ull ? __uint_as_float(v[e + 1]) : 0.f;
                pk[e >> 1] = bf2(d0, d1);
            }
            put_col(sm + S_Y + kt * Y_BYTES, 64, c0, 16, t, pk);
        }
        to_tensor_core();
        if (t == 0) {
            tc_fence_after();
            const uint32_t ig = tc_idesc(128, NG, true), i3 = tc_idesc(128, 16, true);
            for (int k2 = 0; k2 < 2; k2++)
                for (int kk = 0; kk < 4; kk++) {
                    const int acc = (first && k2 == 0 && kk == 0) ? 0 : 1;
                    tc_mma(tmem + C_G, tc_desc(sbase + S_Y + k2 * Y_BYTES + kk * 32),
                           tc_desc(sbase + S_X + k2 * X_BYTES + 64 * TC_ROWB + kk * 32), ig, acc);
                    tc_mma(tmem + C_G3, tc_desc(sbase + S_X + k2 * X_BYTES + kk * 32),
                           tc_desc(sbase + S_Z + k2 * Z_BYTES + kk * 32), i3, acc);
                }
            tc_commit(&mbar);
        }
        if (!(ok = mma_wait())) break;
        first = false;
    }
    if (!ok) {
        if (t == 0 && a.fault) atomicExch(a.fault, 1);
        mbar_wait(&mbar, (phase - 1u) & 1u);              // bounded: let a late MMA finish before freeing
    }
    if (BACK && ok) {
        // this CTA's gradient partial: gW2, gb2 (lanes 0-63), gW1, gb1 (lanes 64-127), gW3
        float* gp = a.gpart + (long long)blockIdx.x * NPARAM;
        const bool any = tile0 < ntiles;
        uint32_t v[16];
        if (warp < 2) {
            const int o = t;
            for (int c0 = 0; c0 < 64; c0 += 16) {
                if (any) { tc_ld16(tl + C_G + c0, v); tc_wait_ld(); }
#pragma unroll
                for (int e = 0; e < 16; e++) gp[OFF_W2 + o * NH + c0 + e] = any ? __uint_as_float(v[e]) : 0.f;
            }
            if (any) { tc_ld16(tl + C_G + 64, v); tc_wait_ld(); }
            gp[OFF_B2 + o] = any ? __uint_as_float(v[NIN]) : 0.f;
            if (any) { tc_ld16(tl + C_G3, v); tc_wait_ld(); }
#pragma unroll
            for (int k = 0; k < NOUT; k++) gp[OFF_W3 + k * NH + o] = any ? __uint_as_float(v[k]) : 0.f;
        } else {
            const int o = t - 64;
            if (any) { tc_ld16(tl + C_G + 64, v); tc_wait_ld(); }
#pragma unroll
            for (int k = 0; k < NIN; k++) gp[OFF_W1 + o * NIN + k] = any ? __uint_as_float(v[k]) : 0.f;
            gp[OFF_B1 + o] = any ? __uint_as_float(v[NIN]) : 0.f;
        }
#pragma unroll
        for (int k = 0; k < NOUT; k++) {
            float s = gb3[k];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
            if (lane == 0) red_b3[warp][k] = s;
        }
        const double ls = warp_sum(loss);
        if (lane == 0) red_l[warp] = ls;
        __syncthreads();
        if (t < NOUT) {
            float s = 0.f;
            for (int w = 0; w < MT / 32; w++) s += red_b3[w][t];
            gp[OFF_B3 + t] = s;
        }
        if (MODE == MLP_TRAIN && t == 0) {
            double s = 0.0;
            for (int w = 0; w < MT / 32; w++) s += red_l[w];
            a.lpart[blockIdx.x] = s * a.inv_npairs;
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) tc_dealloc(tmem, TM_COLS);
}

}  // namespace

int mlp_tc_grid(long long n)
{
    int dev = 0, sms = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const long long tiles = (n + MLP_ROWS - 1) / MLP_ROWS;
    return (int)std::max<long long>(1, std::min<long long>(tiles, sms));
}

cudaError_t mlp_tc_launch(int mode, int grid, cudaStream_t s, const MlpArgs& a)
{
    static bool attr[3] = {false, false, false};
    cudaError_t e = cudaSuccess;
    switch (mode) {
    case MLP_FWD:
        if (!attr[0]) { e = cudaFuncSetAttribute(k_mlp_tc<MLP_FWD>, cudaFuncAttributeMaxDynamicSharedMemorySize, MLP_SMEM); attr[0] = e == cudaSuccess; }
        if (e == cudaSuccess) k_mlp_tc<MLP_FWD><<<grid, MT, MLP_SMEM, s>>>(a);
        break;
    case MLP_BWD:
        if (!attr[1]) { e = cudaFuncSetAttribute(k_mlp_tc<MLP_BWD>, cudaFuncAttributeMaxDynamicSharedMemorySize, MLP_SMEM); attr[1] = e == cudaSuccess; }
        if (e == cudaSuccess) k_mlp_tc<MLP_BWD><<<grid, MT, MLP_SMEM, s>>>(a);
        break;
    default:
        if (!attr[2]) { e = cudaFuncSetAttribute(k_mlp_tc<MLP_TRAIN>, cudaFuncAttributeMaxDynamicSharedMemorySize, MLP_SMEM); attr[2] = e == cudaSuccess; }
        if (e == cudaSuccess) k_mlp_tc<MLP_TRAIN><<<grid, MT, MLP_SMEM, s>>>(a);
        break;
    }
    return e != cudaSuccess ? e : cudaGetLastError();
}

}  // namespace cbg
