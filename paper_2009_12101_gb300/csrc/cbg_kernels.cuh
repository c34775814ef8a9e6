// cbg_kernels.cuh -- CUDA kernels of the restarted Arnoldi step (the Arnoldi step of Fig. 1),
// templated on the basis storage format and on the arithmetic mode.
//
// Data layout in HBM (per solver handle):
//   V       (m+1) columns of codes, column k at V + k*ldb, ldb = ld * bytes(fmt),
//           ld = n rounded up to TILE_ROWS; rows n..ld-1 are zero and stay zero, so every
//           kernel processes whole tiles without bounds checks on the basis.
//   scales  (m+1) FP64 decode factors (sigma_k, 2^e_k or 1)
//   vectors FP64 arrays of ld elements, zero padded.
#pragma once
#include "cbg_device.cuh"
#include "cbg_tma.cuh"

#include <type_traits>

namespace cbg {

constexpr int THREADS = 256;
constexpr int TILE_ROWS = 4096;      // ld (padded rows) is a multiple of this
constexpr int MAXCOLS = 320;         // largest restart length + 1 supported by the kernels
constexpr int DOT_MIN_ROWS = 1024;   // the dot kernel's grid gives every block >= this many rows
constexpr int ARITH_DF32 = 0;
constexpr int ARITH_FP64 = 1;

// Solver state shared by the kernels of one handle (device memory).
struct DevState {
    int active;           // 1 while the current restart cycle continues
    int k;                // Hessenberg columns completed in the cycle
    int stop;             // 0 running, 1 recurrence converged, 2 breakdown, 3 non-finite, 4 kcap
    int kcap;             // steps allowed in this cycle
    int m;                // restart length (leading dimension of H is m+1)
    int record;           // write the residual history
    long long iters;      // Arnoldi steps so far (all cycles)
    long long reorths;
    double bnorm, target; // ||b||, tau ||b||
    double beta, rinf;    // ||r0||_2, ||r0||_inf of the current cycle
    double omega;         // ||A z|| of the current step (omega of Fig. 1)
    double eps_bd;        // breakdown threshold
    double est;           // |g_{j+1}|
    double hn;            // h_{j+1,j}
    long long hist_cap;
    int last_k;           // columns of the previous cycle (set when a cycle starts)
    int fault;            // nonzero: a pipelined kernel gave up waiting (FAULT_TIMEOUT)
    double wnorm, wmax;   // ||w||_2 and ||w||_inf of the orthogonalised w (last axpy block)
    int reorth_now;       // conditional mode: the current step's second pass runs (written at
                          // every step by the first pass's last axpy block, cleared when a
                          // cycle starts)
    int pad_state;
};

// per-handle arrays addressed by the kernels
struct DevArrays {
    DevState* st;
    double* H;            // (m+1) x m raw Hessenberg, column-major
    double* R;            // rotated copy
    double* cs;           // Givens cosines [m]
    double* sn;           // Givens sines   [m]
    double* g;            // rhs of the least-squares problem [m+1]
    double* y;            // solution [m+1] (zero beyond k)
    double* h;            // CGS coefficients, pass 1 [m+1]
    double* u;            // CGS coefficients, pass 2 [m+1]
    double* scales;       // decode scale per basis column [m+1]
    double* hist;         // recurrence residual history (device)
    double* part;         // per-block partial sums [gridmax * (m+2)]
    double* part_norm;    // per-block (sum of squares, max) of the axpy epilogue [gridmax*2]
    double* part_spmv;    // per-block sum of squares and max of SpMV / residual [gridmax*2]
    unsigned int* counters;   // last-block counters (zeroed, reset by the last block)
    int* flag_host;       // mapped host copy of `active` (may be null)
};

// ============================================================================ helpers
// Debug build (-DCBG_DEBUG): a column index outside [0, n) is recorded as FAULT_BOUNDS
// in the solver state and its entry skipped, instead of being read; release builds
// compile the check away (the CSR is validated on the host at create).
__device__ __forceinline__ bool col_ok(int c, long long n, DevState* st)
{
#ifdef CBG_DEBUG
    if ((unsigned long long)(long long)c >= (unsigned long long)n) {
        if (st) atomicExch(&st->fault, FAULT_BOUNDS);
        return false;
    }
#else
    (void)c;
    (void)n;
    (void)st;
#endif
    return true;
}

__device__ __forceinline__ bool last_block(unsigned int* counter)
{
    __shared__ bool is_last;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned int prev = atomicAdd(counter, 1u);
        is_last = (prev == gridDim.x - 1);
    }
    __syncthreads();
    if (is_last) {
        __threadfence();
        if (threadIdx.x == 0) *counter = 0u;   // ready for the next launch
    }
    return is_last;
}

// The last block's sum of squares and maximum over the per-block pairs (part[2b],
// part[2b+1]), b < np (all threads must call it; the results are valid in warp 0):
// thread t adds the pairs t, t + blockDim.x, ... in that order, then block_sum_max folds
// the threads with fixed shuffle trees, so the result depends only on np and
// blockDim.x.  The loads of two pairs are issued before they are added; the maxima of
// the non-negative values are taken on their bit patterns (integer operations).
__device__ __forceinline__ void block_reduce_norm_parts(const double* part, int np, double& ss, double& mx)
{
    __shared__ double rs[32], rm[32];
    const int nt = blockDim.x;
    double s = 0.0;
    unsigned int mh = 0u, ml = 0u;
    for (int p0 = threadIdx.x; p0 < np; p0 += 2 * nt) {
        double vs[2], vm[2];
#pragma unroll
        for (int u = 0; u < 2; u++) {
            const int p = p0 + u * nt;
            vs[u] = p < np ? __ldcg(part + 2 * p) : 0.0;
            vm[u] = p < np ? __ldcg(part + 2 * p + 1) : 0.0;
        }
#pragma unroll
        for (int u = 0; u < 2; u++)
            if (p0 + u * nt < np) {
                s += vs[u];
                const unsigned int h = (unsigned int)__double2hiint(vm[u]), l = (unsigned int)__double2loint(vm[u]);
                if (h > mh || (h == mh && l > ml)) {
                    mh = h;
                    ml = l;
                }
            }
    }
    block_sum_max(s, __hiloint2double((int)mh, (int)ml), rs, rm, ss, mx);
}

// The last block's sums over the per-block partials of nitems items: item i is
// sum_{b < nb} part[b * ldp + i], handed to emit(i, sum) by lane 0 of the warp that
// computed it.  Warp w of nwarps takes the items 2w, 2w + 1, then 2(w + nwarps), ...;
// lane l adds blocks l, l + 32, l + 64, ... in that order and the warp folds its lanes
// with a fixed shuffle tree (the result depends only on nb).  A lane issues the loads of
// eight blocks for both items before adding them, so an item costs about nb / 256 memory
// round trips instead of nb / 32.
template <class Emit>
__device__ __forceinline__ void reduce_block_parts(const double* part, long long ldp, int nb, int nitems, int warp,
                                                   int nwarps, Emit emit)
{
    const int lane = threadIdx.x & 31;
    for (int i0 = 2 * warp; i0 < nitems; i0 += 2 * nwarps) {
        const bool two = i0 + 1 < nitems;
        double s0 = 0.0, s1 = 0.0;
        for (int b0 = 0; b0 < nb; b0 += 256) {
            double v0[8], v1[8];
#pragma unroll
            for (int u = 0; u < 8; u++) {
                const int b = b0 + lane + 32 * u;
                const double* q = part + (long long)b * ldp + i0;
                v0[u] = b < nb ? __ldcg(q) : 0.0;
                v1[u] = b < nb && two ? __ldcg(q + 1) : 0.0;
            }
#pragma unroll
            for (int u = 0; u < 8; u++)
                if (b0 + lane + 32 * u < nb) {
                    s0 += v0[u];
                    s1 += v1[u];
                }
        }
        s0 = warp_sum(s0);
        s1 = warp_sum(s1);
        if (lane == 0) {
            emit(i0, s0);
            if (two) emit(i0 + 1, s1);
        }
    }
}

// FP64 value of element e of a decoded chunk (scale not applied); exact for every format
template <int FMT>
__device__ __forceinline__ double chunk_f64(const uint4& raw, const Chunk<FMT>& ch, int e)
{
    if constexpr (FMT == F64) {
        const unsigned int w[4] = {raw.x, raw.y, raw.z, raw.w};
        return __hiloint2double((int)w[2 * e + 1], (int)w[2 * e]);
    } else if constexpr (SingleFloat<FMT>::value) {
        return f32_to_f64_exact(ch.vh[e]);
    } else {
        return __dadd_rn(f32_to_f64_exact(ch.vh[e]), f32_to_f64_exact(ch.vl[e]));
    }
}

// ============================================================== h = V^T w  (CGS)
// Row-per-lane schedule (the axpy's): a lane owns E consecutive rows (one 16-byte code
// chunk per column) at a time, and the 32 lanes of a warp read 512 contiguous bytes of
// each column.  Every warp runs through its segments once per group of CG columns, keeping one
// double-float accumulator per column (w for its rows is loaded once and reused by the CG
// columns).  The warp then folds the CG accumulators with a transposing butterfly (each
// level halves the columns a lane holds, so CG-1+log2(32/CG) double-float additions per
// lane instead of 5*CG) and parks the column sums in shared memory: warps never wait for
// one another before the end, so their load and compute phases interleave.  The block
// sums its warps in a fixed order, blocks leave per-column partials, and the last block
// to finish adds them in a fixed order (deterministic).
struct DotArgs {
    const unsigned char* V;
    long long ldb;            // bytes per column
    int ncols;
    const int* ncols_dev;     // if non-null, read ncols from device
    const double* scales;
    const double* w;          // FP64 vector, ld elements
    long long nrows;          // ld (multiple of TILE_ROWS)
    double* part;             // [gridDim.x][MAXCOLS]
    unsigned int* counter;
    double* out;              // [ncols]
    const int* active;        // skip when *active == 0 (may be null)
    const float* wdf;         // w split into FP32 pairs, planar: hi[nrows] then lo[nrows] (DF32; may be null)
    // pipelined dot only: waits give up after wait_limit clock cycles (0: the default of
    // about a second); withhold != 0 makes the producer skip its first work item (no
    // arrival, no copies), so that the waits on it run out -- a test of the timeout path
    long long wait_limit;
    int withhold;
};

template <int FMT> struct DotCfg {
    static constexpr int E = 16 / FmtInfo<FMT>::bytes;     // rows per 16-byte chunk
    static constexpr int CG = E >= 16 ? 8 : 16;            // columns per group
};

// One level of the transposing butterfly over N double-float values per lane: lanes with
// bit `o` set keep the upper half, the others the lower half, and each adds its
// partner's copy of the half it keeps.
template <int N>
__device__ __forceinline__ void df_fold_level(float* S, float* C, int lane, int o)
{
    const bool up = (lane & o) != 0;
#pragma unroll
    for (int i = 0; i < N / 2; i++) {
        const float ks = up ? S[i + N / 2] : S[i], kc = up ? C[i + N / 2] : C[i];
        const float ss = up ? S[i] : S[i + N / 2], sc = up ? C[i] : C[i + N / 2];
        const float rs = __shfl_xor_sync(0xffffffffu, ss, o), rc = __shfl_xor_sync(0xffffffffu, sc, o);
        float a = ks, b = kc;
        df_add(a, b, rs, rc);
        S[i] = a;
        C[i] = b;
    }
}
template <int N>
__device__ __forceinline__ void d_fold_level(double* D, int lane, int o)
{
    const bool up = (lane & o) != 0;
#pragma unroll
    for (int i = 0; i < N / 2; i++) {
        const double k = up ? D[i + N / 2] : D[i];
        const double snd = up ? D[i] : D[i + N / 2];
        D[i] = __dadd_rn(k, __shfl_xor_sync(0xffffffffu, snd, o));
    }
}

// Fold CG per-lane sums (CG = 4, 8, 16 or 32) into per-column warp sums.  Returns the
// column (0..CG-1) whose total this lane holds; lanes whose bits below the transposing
// levels (lane & fold_low<CG>()) are zero hold distinct columns (the others hold copies).
template <int CG> __host__ __device__ constexpr int fold_low()
{
    return CG == 32 ? 0 : (CG == 16 ? 1 : (CG == 8 ? 3 : 7));
}

template <int CG>
__device__ __forceinline__ int df_warp_fold(float* S, float* C, int lane)
{
    static_assert(CG == 4 || CG == 8 || CG == 16 || CG == 32, "fold width");
    int col = 0;
    df_fold_level<CG>(S, C, lane, 16);
    col += ((lane >> 4) & 1) * (CG / 2);
    df_fold_level<CG / 2>(S, C, lane, 8);
    col += ((lane >> 3) & 1) * (CG / 4);
    if constexpr (CG >= 8) {
        df_fold_level<CG / 4>(S, C, lane, 4);
        col += ((lane >> 2) & 1) * (CG / 8);
    }
    if constexpr (CG >= 16) {
        df_fold_level<CG / 8>(S, C, lane, 2);
        col += ((lane >> 1) & 1) * (CG / 16);
    }
    if constexpr (CG == 32) {
        df_fold_level<2>(S, C, lane, 1);
        col += lane & 1;
    }
    // the remaining levels are plain butterflies over the one value left
#pragma unroll
    for (int o = (fold_low<CG>() + 1) / 2; o >= 1; o >>= 1) {
        const float rs = __shfl_xor_sync(0xffffffffu, S[0], o), rc = __shfl_xor_sync(0xffffffffu, C[0], o);
        df_add(S[0], C[0], rs, rc);
    }
    return col;
}
template <int CG>
__device__ __forceinline__ int d_warp_fold(double* D, int lane)
{
    static_assert(CG == 4 || CG == 8 || CG == 16, "fold width");
    int col = 0;
    d_fold_level<CG>(D, lane, 16);
    col += ((lane >> 4) & 1) * (CG / 2);
    d_fold_level<CG / 2>(D, lane, 8);
    col += ((lane >> 3) & 1) * (CG / 4);
    if constexpr (CG >= 8) {
        d_fold_level<CG / 4>(D, lane, 4);
        col += ((lane >> 2) & 1) * (CG / 8);
    }
    if constexpr (CG == 16) {
        d_fold_level<2>(D, lane, 2);
        col += (lane >> 1) & 1;
    }
#pragma unroll
    for (int o = (fold_low<CG>() + 1) / 2; o >= 1; o >>= 1) D[0] = __dadd_rn(D[0], __shfl_xor_sync(0xffffffffu, D[0], o));
    return col;
}

// One column group of the dot kernel over the warp's segments.  FULL: all CG columns
// exist (no per-column tests in the streaming loop).
template <int FMT, int ARITH, bool FULL>
__device__ __forceinline__ double dot_group(const DotArgs& a, int c0, int nc, long long sg0, long long nseg,
                                            long long nwt, int lane, int& col)
{
    constexpr int BS = FmtInfo<FMT>::bytes;
    constexpr int E = DotCfg<FMT>::E, CG = DotCfg<FMT>::CG;
    const unsigned char* vbase = a.V + (long long)c0 * a.ldb;
    float2 S2[CG / 2], C2[CG / 2];       // columns (2i, 2i+1) on the packed FP32x2 pipe
    double D[CG];
#pragma unroll
    for (int q = 0; q < CG / 2; q++) { S2[q] = make_float2(0.f, 0.f); C2[q] = make_float2(0.f, 0.f); }
#pragma unroll
    for (int q = 0; q < CG; q++) D[q] = 0.0;
    for (long long sg = sg0; sg < nseg; sg += nwt) {
        const long long row0 = (sg * 32 + lane) * E;
        const unsigned char* p = vbase + row0 * BS;
        uint4 raw[CG];
#pragma unroll
        for (int q = 0; q < CG; q++)
            raw[q] = (FULL || q < nc) ? ldg_stream(p + (long long)q * a.ldb) : make_uint4(0u, 0u, 0u, 0u);
        float wh[E], wl[E];
        double wd[E];
        if (ARITH == ARITH_DF32 && a.wdf) {
            if constexpr (E == 2) {
                const float2 h2 = __ldcg(reinterpret_cast<const float2*>(a.wdf + row0));
                const float2 l2 = __ldcg(reinterpret_cast<const float2*>(a.wdf + a.nrows + row0));
                wh[0] = h2.x; wh[1] = h2.y; wl[0] = l2.x; wl[1] = l2.y;
            } else {
#pragma unroll
                for (int e = 0; e < E; e += 4) {
                    const float4 h4 = __ldcg(reinterpret_cast<const float4*>(a.wdf + row0 + e));
                    const float4 l4 = __ldcg(reinterpret_cast<const float4*>(a.wdf + a.nrows + row0 + e));
                    wh[e] = h4.x; wh[e + 1] = h4.y; wh[e + 2] = h4.z; wh[e + 3] = h4.w;
                    wl[e] = l4.x; wl[e + 1] = l4.y; wl[e + 2] = l4.z; wl[e + 3] = l4.w;
                }
            }
        } else {
#pragma unroll
            for (int e = 0; e < E; e += 2) {
                const double2 w2 = __ldcg(reinterpret_cast<const double2*>(a.w + row0 + e));
                wd[e] = w2.x;
                wd[e + 1] = w2.y;
            }
            if constexpr (ARITH == ARITH_DF32) {
#pragma unroll
                for (int e = 0; e < E; e++) split_f64(wd[e], wh[e], wl[e]);
            }
        }
        if constexpr (ARITH == ARITH_DF32) {
            // a missing column (q >= nc) has zero codes and adds exact zeros
#pragma unroll
            for (int q = 0; q < CG; q += 2) {
                if (!FULL && q >= nc) break;
                Chunk<FMT> c0h, c1h;
                decode_chunk<FMT>(raw[q], c0h);
                decode_chunk<FMT>(raw[q + 1], c1h);
#pragma unroll
                for (int e = 0; e < E; e++) {
                    const float2 wh2 = make_float2(wh[e], wh[e]), nwh2 = make_float2(-wh[e], -wh[e]);
                    const float2 wl2 = make_float2(wl[e], wl[e]);
                    if constexpr (SingleFloat<FMT>::value)
                        df2_mac(S2[q / 2], C2[q / 2], make_float2(c0h.vh[e], c1h.vh[e]), wh2, nwh2, wl2);
                    else
                        df2_mac2(S2[q / 2], C2[q / 2], make_float2(c0h.vh[e], c1h.vh[e]),
                                 make_float2(c0h.vl[e], c1h.vl[e]), wh2, nwh2, wl2);
                }
                df2_renorm(S2[q / 2], C2[q / 2]);
            }
        } else {
#pragma unroll
            for (int q = 0; q < CG; q++) {
                if (!FULL && q >= nc) break;
                Chunk<FMT> ch;
                decode_chunk<FMT>(raw[q], ch);
#pragma unroll
                for (int e = 0; e < E; e++) D[q] = __fma_rn(chunk_f64<FMT>(raw[q], ch, e), wd[e], D[q]);
            }
        }
    }
    if constexpr (ARITH == ARITH_DF32) {
        float S[CG], C[CG];
#pragma unroll
        for (int q = 0; q < CG / 2; q++) {
            S[2 * q] = S2[q].x;
            S[2 * q + 1] = S2[q].y;
            C[2 * q] = C2[q].x;
            C[2 * q + 1] = C2[q].y;
        }
        col = df_warp_fold<CG>(S, C, lane);
        return df_to_double(S[0], C[0]);
    } else {
        col = d_warp_fold<CG>(D, lane);
        return D[0];
    }
}

template <int FMT, int ARITH>
__global__ void __launch_bounds__(THREADS, 2) k_basis_dot(DotArgs a)
{
    if (a.active && *a.active == 0) return;
    constexpr int E = DotCfg<FMT>::E, CG = DotCfg<FMT>::CG;
    constexpr int NW = THREADS / 32;
    constexpr int LOW = fold_low<CG>();            // lane bits below the transposing levels
    __shared__ double red[NW][MAXCOLS];
    const int ncols = a.ncols_dev ? *a.ncols_dev : a.ncols;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;

    // warp segments of 32 chunks (32*E rows), dealt round-robin in SM-spread order:
    // warp w of block b takes segments w*gridDim.x + b + k*(all warps), so at any time the
    // GPU streams one contiguous window of each column, and the last, partial round is
    // shared by the blocks of every SM.  Warps never wait for one another until the end.
    const long long nseg = a.nrows / (32 * E);
    const long long nwt = (long long)gridDim.x * NW;
    const long long sg0 = (long long)warp * gridDim.x + blockIdx.x;

    for (int c0 = 0; c0 < ncols; c0 += CG) {
        const int nc = ncols - c0 < CG ? ncols - c0 : CG;
        int col;
        const double wsum = nc == CG ? dot_group<FMT, ARITH, true>(a, c0, nc, sg0, nseg, nwt, lane, col)
                                     : dot_group<FMT, ARITH, false>(a, c0, nc, sg0, nseg, nwt, lane, col);
        // the warp's column sums wait in shared memory for the block sum
        if ((lane & LOW) == 0 && col < nc) red[warp][c0 + col] = wsum;
    }
    __syncthreads();
    // the block's warps in a fixed order
    for (int col = threadIdx.x; col < ncols; col += THREADS) {
        double tot = 0.0;
#pragma unroll
        for (int w = 0; w < NW; w++) tot += red[w][col];
        a.part[(long long)blockIdx.x * MAXCOLS + col] = tot;
    }

    if (last_block(a.counter))
        reduce_block_parts(a.part, MAXCOLS, gridDim.x, ncols, warp, NW,
                           [&](int col, double sum) { a.out[col] = sum * a.scales[col]; });
}

// ====================================================== w_out = w_in + sum_k V_k c_k
// c_k = sign * scales[k] * coef[k].  Row-per-lane schedule: a lane owns E consecutive
// rows at a time, reads 16 B of every column (512 contiguous bytes across the warp) and
// keeps E double-float accumulators; warps take 32-chunk segments round-robin in
// SM-spread order (as in the dot kernel).  Epilogue modes:
//   EPI_SUB   w_out = w_in - V coef, plus per-block sum of squares and max |w_out|
//   EPI_XUPD  x += dinv .* (V coef) (dinv may be null), x = w_out, w_in unused
//   EPI_PLAIN w_out = V coef
constexpr int EPI_SUB = 0, EPI_XUPD = 1, EPI_PLAIN = 2;

struct AxpyArgs {
    const unsigned char* V;
    long long ldb;
    int ncols;
    const int* ncols_dev;
    const double* scales;
    const double* coef;       // device [ncols]
    double sign;
    const double* w_in;
    double* w_out;            // EPI_SUB, DF32: may be null when wdf_out is set (only the split
                              // copy is written; no norms then, counter must be null)
    const double* dinv;       // Jacobi (EPI_XUPD), may be null
    long long nrows;          // ld
    long long n;              // true rows (norms exclude padding)
    double* part_norm;        // [gridDim.x][2]
    const int* active;
    unsigned int* counter;    // EPI_SUB final pass: last block writes st->wnorm, st->wmax
    DevState* st;
    float* wdf_out;           // EPI_SUB: also store w_out split, planar hi[nrows] then lo[nrows] (may be null)
    const float* wdf_in;      // EPI_SUB, DF32: w_in given as such planes instead (may be null; may equal wdf_out)
    int* reorth_flag;         // EPI_SUB with counter, conditional re-orthogonalisation (Fig. 1): the
    double eta;               //   last block sets *reorth_flag = (||w_out|| < eta * st->omega)
};

// Blocks per SM asked of the register allocator: 4 for 8-byte codes (measured 5 % faster
// than 3), 3 for 2- and 4-byte codes (4 was slower for f32), 2 for 1-byte codes.
template <int FMT, int ARITH, int EPI>
__global__ void __launch_bounds__(THREADS, FmtInfo<FMT>::bytes >= 8 ? 4 : (FmtInfo<FMT>::bytes >= 2 ? 3 : 2)) k_basis_axpy(AxpyArgs a)
{
    if (a.active && *a.active == 0) return;
    constexpr int BS = FmtInfo<FMT>::bytes;
    constexpr int E = 16 / BS;
    constexpr int U = E <= 8 ? 8 : 4;   // columns (16-byte loads) in flight per thread
    __shared__ float2 cs[MAXCOLS];
    __shared__ double red_s[THREADS / 32], red_m[THREADS / 32];
    const int ncols = a.ncols_dev ? *a.ncols_dev : a.ncols;
    for (int k = threadIdx.x; k < ncols; k += THREADS) {
        double c = a.sign * a.scales[k] * a.coef[k];
        float2 s;
        if constexpr (ARITH == ARITH_DF32) split_f64(c, s.x, s.y);
        else s = *reinterpret_cast<float2*>(&c);
        cs[k] = s;
    }
    __syncthreads();

    double ss = 0.0;             // epilogue partials: sum of squares (FP64; double-float in
    float ssS = 0.f, ssC = 0.f;  // (ssS, ssC) with DF32 arithmetic) and
    unsigned int mxh = 0, mxl = 0;   // max |w| as the bit pattern of a non-negative double
                                     // (high and low words, compared with 32-bit operations)
    // warp segments of 32 chunks (32*E rows), dealt round-robin in SM-spread order
    const long long nseg = a.nrows / (32 * E);
    const long long nwt = (long long)gridDim.x * (THREADS / 32);
    // The segment loop, compiled per epilogue case so that no case carries the others'
    // instructions as predicated code (on GB300 a predicated-off FP64-pipe instruction
    // still occupies the narrow FP64 pipe): M = 1 the split planes only, M = 2 w and its
    // norms without the split copy (the final CGS pass), M = 0 any combination.
    auto segments = [&](auto mode_tag) {
        constexpr int M = decltype(mode_tag)::value;
        (void)M;
        for (long long sg = (long long)(threadIdx.x >> 5) * gridDim.x + blockIdx.x; sg < nseg; sg += nwt) {
            const long long row0 = (sg * 32 + (threadIdx.x & 31)) * E;
            const unsigned char* base = a.V + row0 * BS;
            // rows of this lane below n (the norms exclude the padding), as a 32-bit count
            const int nvalid = a.n - row0 >= E ? E : (a.n > row0 ? (int)(a.n - row0) : 0);
            (void)nvalid;
            float2 S2[E / 2], C2[E / 2];     // rows (2i, 2i+1) on the packed FP32x2 pipe
            double D[E];
#pragma unroll
            for (int e = 0; e < E / 2; e++) { S2[e] = make_float2(0.f, 0.f); C2[e] = make_float2(0.f, 0.f); }
#pragma unroll
            for (int e = 0; e < E; e++) D[e] = 0.0;
            auto column = [&](const uint4& raw, float2 c) {
                Chunk<FMT> ch;
                decode_chunk<FMT>(raw, ch);
                if constexpr (ARITH == ARITH_DF32) {
                    const float2 ch2 = make_float2(c.x, c.x), nch2 = make_float2(-c.x, -c.x), cl2 = make_float2(c.y, c.y);
#pragma unroll
                    for (int e = 0; e < E; e += 2) {
                        if constexpr (SingleFloat<FMT>::value)
                            df2_mac(S2[e / 2], C2[e / 2], make_float2(ch.vh[e], ch.vh[e + 1]), ch2, nch2, cl2);
                        else
                            df2_mac2(S2[e / 2], C2[e / 2], make_float2(ch.vh[e], ch.vh[e + 1]),
                                     make_float2(ch.vl[e], ch.vl[e + 1]), ch2, nch2, cl2);
                    }
                } else {
                    const double cd = *reinterpret_cast<double*>(&c);
#pragma unroll
                    for (int e = 0; e < E; e++) D[e] = __fma_rn(chunk_f64<FMT>(raw, ch, e), cd, D[e]);
                }
            };
            int k = 0;
            if constexpr (ARITH == ARITH_DF32 && BS == 4) {
                // 4-byte codes (latency-bound): two groups of four columns, software-pipelined,
                // so the next group's loads are in flight while the current group is
                // accumulated (measured 3 % faster for f32; slower for the FMA-bound 2-byte codes)
                constexpr int H = 4;
                uint4 ra[H], rb[H];
                if (H <= ncols) {
#pragma unroll
                    for (int q = 0; q < H; q++) ra[q] = ldg_stream(base + (long long)q * a.ldb);
                }
                for (; k + 2 * H <= ncols; k += 2 * H) {
#pragma unroll
                    for (int q = 0; q < H; q++) rb[q] = ldg_stream(base + (long long)(k + H + q) * a.ldb);
#pragma unroll
                    for (int q = 0; q < H; q++) column(ra[q], cs[k + q]);
#pragma unroll
                    for (int e = 0; e < E / 2; e++) df2_renorm(S2[e], C2[e]);
                    if (k + 3 * H <= ncols) {
#pragma unroll
                        for (int q = 0; q < H; q++) ra[q] = ldg_stream(base + (long long)(k + 2 * H + q) * a.ldb);
                    }
#pragma unroll
                    for (int q = 0; q < H; q++) column(rb[q], cs[k + H + q]);
#pragma unroll
                    for (int e = 0; e < E / 2; e++) df2_renorm(S2[e], C2[e]);
                }
                if (k + H <= ncols) {             // a last full group of four (already loaded)
#pragma unroll
                    for (int q = 0; q < H; q++) column(ra[q], cs[k + q]);
#pragma unroll
                    for (int e = 0; e < E / 2; e++) df2_renorm(S2[e], C2[e]);
                    k += H;
                }
            } else {
                for (; k + U <= ncols; k += U) {
                    uint4 raw[U];
#pragma unroll
                    for (int q = 0; q < U; q++) raw[q] = ldg_stream(base + (long long)(k + q) * a.ldb);
#pragma unroll
                    for (int q = 0; q < U; q++) {
                        column(raw[q], cs[k + q]);
                        if constexpr (ARITH == ARITH_DF32) {
                            if ((q & 3) == 3) {
#pragma unroll
                                for (int e = 0; e < E / 2; e++) df2_renorm(S2[e], C2[e]);
                            }
                        }
                    }
                }
            }
            for (; k < ncols; k++) column(ldg_stream(base + (long long)k * a.ldb), cs[k]);
            float S[E], C[E];
#pragma unroll
            for (int e = 0; e < E / 2; e++) {
                S[2 * e] = S2[e].x;
                S[2 * e + 1] = S2[e].y;
                C[2 * e] = C2[e].x;
                C[2 * e + 1] = C2[e].y;
            }
            // epilogue
#pragma unroll
            for (int e = 0; e < E; e++) {
                const long long i = row0 + e;
                double acc;
                if constexpr (ARITH == ARITH_DF32) {
                    if constexpr (EPI == EPI_SUB) {
                        float wh, wl;
                        if (a.wdf_in) {
                            wh = a.wdf_in[i];
                            wl = a.wdf_in[a.nrows + i];
                        } else {
                            split_f64(a.w_in[i], wh, wl);
                        }
                        df_add(S[e], C[e], wh, wl);
                    }
                    if (M == 1 || (M == 0 && EPI == EPI_SUB && !a.w_out)) {
                        // only the split copy is wanted (the first CGS pass when the second
                        // always runs): the renormalised pair itself, no FP64 operation, no norms
                        float h, l;
                        two_sum(S[e], C[e], h, l);
                        a.wdf_out[i] = h;
                        a.wdf_out[a.nrows + i] = l;
                        continue;
                    }
                    if constexpr (EPI == EPI_SUB) {
                        // sum of squares in double-float on the FP32 pipe (GB300's FP64 pipe
                        // runs at about 1/70 of it): (h + l)^2 = h^2 + 2hl, h^2 exact as a pair
                        float h, l;
                        two_sum(S[e], C[e], h, l);
                        if ((M == 2 || (M == 0 && a.counter)) && e < nvalid) {
                            const float p = __fmul_rn(h, h);
                            float q = __fmaf_rn(h, h, -p);
                            q = __fmaf_rn(__fadd_rn(h, h), l, q);
                            const float t = __fadd_rn(ssS, p), bb = __fsub_rn(t, ssS);
                            ssC = __fadd_rn(ssC, __fadd_rn(__fadd_rn(__fsub_rn(ssS, __fsub_rn(t, bb)), __fsub_rn(p, bb)), q));
                            ssS = t;
                        }
                        acc = df_to_double(h, l);
                    } else {
                        acc = df_to_double(S[e], C[e]);
                    }
                } else {
                    acc = D[e];
                    if constexpr (EPI == EPI_SUB) acc = __dadd_rn(a.w_in[i], acc);
                }
                if constexpr (EPI == EPI_SUB) {
                    a.w_out[i] = acc;
                    if (M == 0 && a.wdf_out) {
                        float h, l;
                        split_f64(acc, h, l);
                        a.wdf_out[i] = h;
                        a.wdf_out[a.nrows + i] = l;
                    }
                    if ((M == 2 || (M == 0 && a.counter)) && e < nvalid) {   // the norms only when a last block reads them
                        if constexpr (ARITH != ARITH_DF32) ss = __fma_rn(acc, acc, ss);
                        const unsigned int ah = (unsigned int)__double2hiint(acc) & 0x7FFFFFFFu;
                        const unsigned int al = (unsigned int)__double2loint(acc);
                        if (ah > mxh || (ah == mxh && al > mxl)) {
                            mxh = ah;
                            mxl = al;
                        }
                    }
                } else if constexpr (EPI == EPI_XUPD) {
                    if (i < a.n) {
                        double d = a.dinv ? __dmul_rn(a.dinv[i], acc) : acc;
                        a.w_out[i] = __dadd_rn(a.w_out[i], d);
                    }
                } else {
                    a.w_out[i] = acc;
                }
            }
        }
    };
    if constexpr (EPI == EPI_SUB && ARITH == ARITH_DF32) {
        if (!a.w_out) segments(std::integral_constant<int, 1>{});
        else if (!a.wdf_out && a.counter) segments(std::integral_constant<int, 2>{});
        else segments(std::integral_constant<int, 0>{});
    } else {
        segments(std::integral_constant<int, 0>{});
    }
    if constexpr (EPI == EPI_SUB) {
        if (!a.counter) return;
        if constexpr (ARITH == ARITH_DF32) ss = df_to_double(ssS, ssC);
        double s, m;
        block_sum_max(ss, __hiloint2double((int)mxh, (int)mxl), red_s, red_m, s, m);
        if (threadIdx.x == 0) {
            a.part_norm[2 * blockIdx.x] = s;
            a.part_norm[2 * blockIdx.x + 1] = m;
        }
        {
            if (last_block(a.counter)) {
                double s2, m2;
                block_reduce_norm_parts(a.part_norm, gridDim.x, s2, m2);
                if (threadIdx.x == 0) {
                    const double wn = sqrt(s2);
                    a.st->wnorm = wn;
                    a.st->wmax = m2;
                    if (a.reorth_flag) *a.reorth_flag = wn < a.eta * a.st->omega ? 1 : 0;
                }
            }
        }
    }
}

// ========================================== store v_{j+1} = w / h_{j+1,j} (basis extension)
// Every block reads the norms finalised by the preceding axpy, forms h_{j+1,j}, 1/h and
// the format's scale, and encodes its rows into column `col`.  The last block to finish
// additionally completes the Hessenberg column j (h from pass 1 plus u from pass 2),
// applies the Givens rotations (Section 2), updates g, writes the residual history and
// decides whether the cycle continues.
// mode 0: Arnoldi step (finalize + store column j+1); mode 1: first vector of a cycle
// (w = r0, norms from the residual kernel, no Hessenberg work).
struct StoreArgs {
    DevArrays d;
    const double* w;
    unsigned char* Vcol;      // destination column
    int col;                  // index of the destination column (scale slot)
    int j;                    // Hessenberg column being completed (mode 0)
    int mode;
    int reorth;               // pass 2 ran (h += u)
    long long n;
    int fmt;
    unsigned int* counter;    // last-block counter (mode 0: the last block runs the finalize)
    int hexp;                 // mode 0: the column (h, ||w||) came from the operator scaled by
                              // 2^-hexp; the Hessenberg column is it times 2^hexp (0: as is)
    const int* reorth_dev;    // conditional mode: device flag replacing `reorth`; when it is 0
    const double* w_alt;      //   the vector to store is w_alt (the first pass's output)
};


// Executed by warp 0 of the store kernel's block 0.  The column, the previous
// rotations and the coefficients are staged in shared memory by the whole warp first.
//
// Applying the j previous rotations to the new column is a first-order linear recurrence
// in the carried entry x (x_0 = h_0, x_{i+1} = -s_i x_i + c_i h_{i+1}, rotated entry
// R_i = c_i x_i + s_i h_{i+1}).  GB300's FP64 unit has a long latency, so instead of a
// j-long dependent chain the warp evaluates it as a scan of affine maps: each lane
// composes the maps of a contiguous chunk of rotations, an exclusive warp scan composes
// the chunks, and each lane then replays its chunk from its incoming x.  The chain is
// 2*ceil(j/32) + 5 compositions long.
static __device__ void arnoldi_finalize(const StoreArgs& a, double hn, double* sR, double* sRo, double* scs,
                                        double* ssn)
{
    DevState* st = a.d.st;
    const int j = a.j;
    const int lane = threadIdx.x & 31;
    // every state field the warp needs, loaded together before anything is written (the
    // stores below would otherwise order each later load behind them: one L2 round trip each)
    const int ldh = st->m + 1;
    const int reorth = a.reorth_dev ? *a.reorth_dev : a.reorth;   // did the second pass run
    const double omega_raw = st->omega, eps_bd = st->eps_bd, target = st->target, bnorm = st->bnorm;
    const int kcap = st->kcap, record = st->record;
    const long long iters = st->iters, reorths = st->reorths, hist_cap = st->hist_cap;
    const double gj = a.d.g[j];
    // back from the power-of-two normalised operator (exact); hn and omega are scaled
    // after the staging loads are issued, so that those do not wait for the state loads
    const double hs = a.hexp ? pow2d(a.hexp) : 1.0;
    // up to 128 entries per round: all of a round's loads are issued before the first of
    // them is used (issued one entry at a time, every entry cost an L2 round trip)
    for (int base = lane; base <= j + 1; base += 128) {
        double hv[4], uv[4], cv[4], sv[4];
#pragma unroll
        for (int q = 0; q < 4; q++) {
            const int i = base + 32 * q;
            hv[q] = i <= j ? __ldcg(a.d.h + i) : 0.0;
            uv[q] = i <= j ? __ldcg(a.d.u + i) : 0.0;   // read always, added only after pass 2
            cv[q] = i < j ? a.d.cs[i] : 0.0;
            sv[q] = i < j ? a.d.sn[i] : 0.0;
        }
#pragma unroll
        for (int q = 0; q < 4; q++) {
            const int i = base + 32 * q;
            if (i > j + 1) break;
            double v = __dmul_rn(hn, hs);
            if (i <= j) {
                v = hv[q];
                if (reorth) v = __dadd_rn(v, uv[q]);
                v = __dmul_rn(v, hs);
            }
            sR[i] = v;
            if (i < j) {
                scs[i] = cv[q];
                ssn[i] = sv[q];
            }
        }
    }
    __syncwarp();
    hn = __dmul_rn(hn, hs);
    const double omega = __dmul_rn(omega_raw, hs);
    double* Hc = a.d.H + (long long)j * ldh;
    for (int i = lane; i < ldh; i += 32) Hc[i] = i <= j + 1 ? sR[i] : 0.0;   // raw column
    __syncwarp();
    // chunk [i0, i1) of the rotations for this lane; the rotated entries go to sRo (not in
    // place: a neighbouring lane still reads the unrotated h_{i+1})
    const int K = (j + 31) / 32;
    const int i0 = lane * K < j ? lane * K : j, i1 = i0 + K < j ? i0 + K : j;
    double A = 1.0, B = 0.0;                 // composite map x -> A x + B of the chunk
    for (int i = i0; i < i1; i++) {
        const double ai = -ssn[i], bi = __dmul_rn(scs[i], sR[i + 1]);
        B = __fma_rn(ai, B, bi);
        A = __dmul_rn(ai, A);
    }
    // exclusive scan of the chunk maps: (A, B) of lanes 0 .. lane-1, composed in order
    double PA = A, PB = B;                   // inclusive prefix
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const double qa = __shfl_up_sync(0xffffffffu, PA, o), qb = __shfl_up_sync(0xffffffffu, PB, o);
        if (lane >= o) {                     // (PA, PB) o (qa, qb): x -> PA (qa x + qb) + PB
            PB = __fma_rn(PA, qb, PB);
            PA = __dmul_rn(PA, qa);
        }
    }
    double EA = __shfl_up_sync(0xffffffffu, PA, 1), EB = __shfl_up_sync(0xffffffffu, PB, 1);
    if (lane == 0) { EA = 1.0; EB = 0.0; }
    double x = __fma_rn(EA, sR[0], EB);      // carried entry entering this lane's chunk
    for (int i = i0; i < i1; i++) {
        const double c = scs[i], sn = ssn[i], h1 = sR[i + 1];
        sRo[i] = __dadd_rn(__dmul_rn(c, x), __dmul_rn(sn, h1));
        x = __dadd_rn(__dmul_rn(-sn, x), __dmul_rn(c, h1));
    }
    __syncwarp();
    // the lane that applied rotation j-1 holds the carried entry after all of them
    const int last = j > 0 ? (j - 1) / K : 0;
    const double r0all = __shfl_sync(0xffffffffu, x, last);
    if (lane == 0) {
        const double r0 = j > 0 ? r0all : sR[0];
        double rr = hypot(r0, hn);
        double c, s;
        if (rr == 0.0) { c = 1.0; s = 0.0; }
        else {                               // one FP64 division on the critical chain, not two
            const double ri = 1.0 / rr;
            c = __dmul_rn(r0, ri);
            s = __dmul_rn(hn, ri);
        }
        a.d.cs[j] = c;
        a.d.sn[j] = s;
        sRo[j] = rr;
        sRo[j + 1] = 0.0;
        double gn = __dmul_rn(-s, gj);
        a.d.g[j + 1] = gn;
        a.d.g[j] = __dmul_rn(c, gj);
        double est = fabs(gn);
        st->est = est;
        st->hn = hn;
        st->k = j + 1;
        st->iters = iters + 1;
        if (reorth) st->reorths = reorths + 1;
        if (record && iters + 1 <= hist_cap) a.d.hist[iters] = est / bnorm;
        int stop = 0;
        if (!isfinite(hn) || !isfinite(omega) || !isfinite(est)) stop = 3;
        else if (!(hn > eps_bd * omega)) stop = 2;
        else if (est <= target) stop = 1;
        else if (j + 1 >= kcap) stop = 4;
        if (stop) {
            st->stop = stop;
            st->active = 0;
            if (a.d.flag_host) *(volatile int*)a.d.flag_host = 0;
        }
    }
    __syncwarp();
    double* Rc = a.d.R + (long long)j * ldh;
    for (int i = lane; i < ldh; i += 32) Rc[i] = i <= j + 1 ? sRo[i] : 0.0;
}

template <int FMT>
__global__ void __launch_bounds__(THREADS, 4) k_store(StoreArgs a)
{
    DevState* st = a.d.st;
    if (st->active == 0) return;
    __shared__ double sh_inv;
    __shared__ EncParams sh_ep;
    __shared__ double sR[MAXCOLS + 1], sRo[MAXCOLS + 1], scs[MAXCOLS], ssn[MAXCOLS];
    // Mode 0: block 0 completes the Hessenberg column and the Givens update (a serial
    // chain of FP64 operations on one warp) while blocks 1.. encode the new basis vector:
    // the chain needs only h, u and ||w||, all known when the kernel starts, so its warp
    // starts at once.  Block 0 is dispatched first, so it never waits for an encoding
    // block to leave the SM.
    if (a.mode == 0 && blockIdx.x == 0) {
        if (threadIdx.x < 32) arnoldi_finalize(a, st->wnorm, sR, sRo, scs, ssn);
        return;
    }
    if (threadIdx.x == 0) {
        // norms of the vector to store: the residual (first vector of a cycle) or the
        // orthogonalised w, both finalised by the last block of the producing kernel
        const double hn = a.mode == 1 ? st->beta : st->wnorm;
        const double mx = a.mode == 1 ? st->rinf : st->wmax;
        const double inv = 1.0 / hn;
        sh_inv = inv;
        sh_ep = enc_params(FMT, __dmul_rn(mx, inv));
    }
    __syncthreads();
    const int eb = a.mode == 0 ? (int)blockIdx.x - 1 : (int)blockIdx.x;     // encoding block
    const int neb = a.mode == 0 ? (int)gridDim.x - 1 : (int)gridDim.x;
    const double inv = sh_inv;
    const EncParams ep = sh_ep;
    if (eb == 0 && threadIdx.x == 0) a.d.scales[a.col] = ep.scale;
    const double* wsrc = (a.reorth_dev && *a.reorth_dev == 0) ? a.w_alt : a.w;
    const long long stride = (long long)neb * THREADS;
    for (long long i0 = (long long)eb * THREADS + threadIdx.x; i0 < a.n; i0 += 4 * stride) {
        double wv[4];
#pragma unroll
        for (int q = 0; q < 4; q++) {   // four loads in flight per thread
            const long long i = i0 + q * stride;
            wv[q] = i < a.n ? __ldcg(wsrc + i) : 0.0;
        }
#pragma unroll
        for (int q = 0; q < 4; q++) {
            const long long i = i0 + q * stride;
            if (i < a.n) encode_store<FMT>(a.Vcol, i, __dmul_rn(wv[q], inv), ep);
        }
    }
}

// ======================================================= SpMV with on-the-fly decode
// y = A x (x FP64) or y = A dec(code column) (the Arnoldi SpMV of Fig. 1; right preconditioning with
// Jacobi is folded into the stored values A D^{-1}).  GROUP lanes per CSR row.  The
// per-block sum of squares and max |y| of the owned rows go to part; in residual mode
// y = b - A x.  The last block turns the partials into omega (Arnoldi mode) or beta /
// ||r||_inf and the cycle's active flag (residual mode).
constexpr int SPMV_ARNOLDI = 0, SPMV_RESIDUAL = 1, SPMV_PLAIN = 2, SPMV_ACCUM = 3;

struct SpmvArgs {
    const int* rowptr;
    const int* col;
    const double* val;
    const void* x;            // FP64 vector or code column
    double xscale;
    const double* xscale_dev; // per-column scale on device (Arnoldi mode)
    const double* b;          // residual mode
    double* y;
    long long n;
    double* part;             // [gridDim.x][2]
    unsigned int* counter;
    DevState* st;             // Arnoldi: omega; residual: beta, rinf, active
    int* flag_host;
    const int* active;
    float* ydf;               // Arnoldi: also store y split, planar hi[ydf_ld] then lo (may be null)
    long long ydf_ld;
    // Arnoldi: the values split into FP32 hi[nnz] then lo[nnz] planes; when set, the row
    // products are formed and summed in double-float instead of FP64, y is delivered only
    // as its (renormalised) double-float planes ydf (required then) and omega = ||y|| is
    // summed in double-float (may be null)
    const float* valdf;
    long long nnz;
    // Arnoldi, FP64 rows: y = 2^xexp A x, the operator normalised by a power of two (the
    // split planes valdf hold it already scaled)
    int xexp;
};

template <int XFMT, int GROUP, int MODE>
__global__ void __launch_bounds__(THREADS) k_spmv(SpmvArgs a)
{
    if (MODE == SPMV_ARNOLDI && a.active && *a.active == 0) return;
    __shared__ double red_s[THREADS / 32], red_m[THREADS / 32];
    const int lane_g = threadIdx.x & (GROUP - 1);
    const long long gid = ((long long)blockIdx.x * THREADS + threadIdx.x) / GROUP;
    const long long ngroups = (long long)gridDim.x * THREADS / GROUP;
    double xs = a.xscale_dev ? *a.xscale_dev : a.xscale;
    if (a.xexp) xs = __dmul_rn(xs, pow2d(a.xexp));
    double ss = 0.0;
    unsigned long long mxb = 0;
    auto xval = [&](int c) -> double {
        if constexpr (XFMT < 0) return reinterpret_cast<const double*>(a.x)[c];
        else return code_value<XFMT>(a.x, c);
    };
    // row epilogue: scale, residual / accumulate, store (and the split copy), norms
    auto finish = [&](long long row, double s) {
        if constexpr (XFMT >= 0) {
            if (xs != 1.0) s = __dmul_rn(s, xs);   // unit scale (float formats): no FP64 op
        }
        double yv = s;
        if constexpr (MODE == SPMV_RESIDUAL) yv = __dsub_rn(a.b[row], s);
        if constexpr (MODE == SPMV_ACCUM) yv = __dadd_rn(a.y[row], s);
        a.y[row] = yv;
        if constexpr (MODE == SPMV_ARNOLDI) {
            if (a.ydf) {
                float h, l;
                split_f64(yv, h, l);
                a.ydf[row] = h;
                a.ydf[a.ydf_ld + row] = l;
            }
        }
        ss = __fma_rn(yv, yv, ss);
        // max |y| on the bit patterns of non-negative doubles (integer pipe)
        const unsigned long long ab = (unsigned long long)__double_as_longlong(yv) & 0x7FFFFFFFFFFFFFFFull;
        mxb = ab > mxb ? ab : mxb;
    };
    // double-float row products (Arnoldi mode, split values): every product val * x is
    // formed exactly as an FP32 pair (TwoProd) and summed with TwoSum, so the FP64 pipe
    // only converts the row result; otherwise one FP64 FMA per nonzero
    const bool dfrows = MODE == SPMV_ARNOLDI && a.valdf != nullptr;
    constexpr bool XEXACT = XFMT == F32 || XFMT == F16 || XFMT == BF16 || XFMT == E4M3 || XFMT == I16;
    auto dfadd = [](float& S, float& C, float pr, float er) {   // (S, C) += pr + er
        const float t = __fadd_rn(S, pr), bb = __fsub_rn(t, S);
        C = __fadd_rn(C, __fadd_rn(__fadd_rn(__fsub_rn(S, __fsub_rn(t, bb)), __fsub_rn(pr, bb)), er));
        S = t;
    };
    float ssS = 0.f, ssC = 0.f, xsh = 1.f, xsl = 0.f;    // double-float rows: ||y||^2, scale
    const bool xsplit = dfrows && xs != 1.0;
    if (xsplit) split_f64(xs, xsh, xsl);
    const float* vlo = dfrows ? a.valdf + a.nnz : nullptr;       // lo plane of the values
    float* ylo = dfrows ? a.ydf + a.ydf_ld : nullptr;            // lo plane of w
    // the row loop, compiled twice: once with the double-float products and once with
    // FP64 FMAs, so neither path carries the other's instructions (predicated FP64-pipe
    // instructions would still occupy GB300's narrow FP64 pipe)
    auto rows = [&](auto df_tag) {
        constexpr bool DF = decltype(df_tag)::value;
        // 32-bit row arithmetic: CSR indices are int32, so n < 2^31 and row + ngroups
        // stays below 2^32
        const unsigned int n32 = (unsigned int)a.n, ng32 = (unsigned int)ngroups;
        for (unsigned int row = (unsigned int)gid;; row += ng32) {
            const bool valid = row < n32;
            if constexpr (GROUP > 1) {
                if (__all_sync(0xFFFFFFFFu, !valid)) break;   // warp-uniform exit around shuffles
            } else {
                if (!valid) break;
            }
            const int p0 = valid ? a.rowptr[row] : 0, p1 = valid ? a.rowptr[row + 1] : 0;
            double s = 0.0;
            if constexpr (DF) {
                float S = 0.f, C = 0.f;
                for (int p = p0 + lane_g; p < p1; p += GROUP) {
                    const float vh = a.valdf[p], vl = vlo[p];
                    const int cp = a.col[p];
                    if (!col_ok(cp, a.n, a.st)) continue;
                    float xh, xl;
                    xval_df<XFMT>(a.x, cp, xh, xl);
                    const float pr = __fmul_rn(vh, xh);
                    float er = __fmaf_rn(vh, xh, -pr);           // exact product error
                    er = __fmaf_rn(vl, xh, er);
                    if constexpr (!XEXACT) er = __fmaf_rn(vh, xl, er);
                    dfadd(S, C, pr, er);
                }
                if constexpr (GROUP > 1) {
#pragma unroll
                    for (int o = GROUP / 2; o > 0; o >>= 1) {
                        const float S2 = __shfl_xor_sync(0xFFFFFFFFu, S, o), C2 = __shfl_xor_sync(0xFFFFFFFFu, C, o);
                        const float t = __fadd_rn(S, S2), bb = __fsub_rn(t, S);
                        C = __fadd_rn(__fadd_rn(C, C2), __fadd_rn(__fsub_rn(S, __fsub_rn(t, bb)), __fsub_rn(S2, bb)));
                        S = t;
                    }
                }
                if (valid && lane_g == 0) {
                    float hi, lo;
                    two_sum(S, C, hi, lo);                       // renormalise
                    if (xsplit) {                                // integer / power-of-two scales
                        const float p = __fmul_rn(hi, xsh);
                        float e = __fmaf_rn(hi, xsh, -p);
                        e = __fmaf_rn(hi, xsl, e);
                        e = __fmaf_rn(lo, xsh, e);
                        two_sum(p, e, hi, lo);
                    }
                    a.ydf[row] = hi;
                    ylo[row] = lo;
                    const float p = __fmul_rn(hi, hi);           // ||y||^2 in double-float
                    float e = __fmaf_rn(hi, hi, -p);
                    e = __fmaf_rn(__fadd_rn(hi, hi), lo, e);
                    dfadd(ssS, ssC, p, e);
                }
                continue;
            } else {
                for (int p = p0 + lane_g; p < p1; p += GROUP) {
                    const int cp = a.col[p];
                    if (col_ok(cp, a.n, a.st)) s = __fma_rn(a.val[p], xval(cp), s);
                }
                if constexpr (GROUP > 1) {
#pragma unroll
                    for (int o = GROUP / 2; o > 0; o >>= 1) s += __shfl_xor_sync(0xFFFFFFFFu, s, o);
                }
            }
            if (valid && lane_g == 0) finish(row, s);
        }
    };
    if (dfrows) rows(std::true_type{});
    else rows(std::false_type{});
    const double mx = __longlong_as_double((long long)mxb);
    if constexpr (MODE == SPMV_PLAIN || MODE == SPMV_ACCUM) return;
    else {
        if (dfrows) ss = df_to_double(ssS, ssC);
        double s, m;
        block_sum_max(ss, mx, red_s, red_m, s, m);
        if (threadIdx.x == 0) {
            a.part[2 * blockIdx.x] = s;
            a.part[2 * blockIdx.x + 1] = m;
        }
        if (last_block(a.counter)) {
            {
                double s2, m2;
                block_reduce_norm_parts(a.part, gridDim.x, s2, m2);
                if (threadIdx.x == 0) {
                    DevState* st = a.st;
                    if (MODE == SPMV_ARNOLDI) {
                        st->omega = sqrt(s2);
                    } else {
                        st->beta = sqrt(s2);
                        st->rinf = m2;
                    }
                }
            }
        }
    }
}

// ================================================== SpMV on a sliced-ELL copy of the matrix
// The per-step SpMV (Arnoldi mode, double-float rows) on the matrix re-laid out in chunks
// of 32 consecutive rows (sliced ELLPACK with slice 32): chunk c holds len[c] = the
// longest row of the chunk, entry k of the chunk's row `lane` at off[c] + 32 k + lane
// (shorter rows padded with zero values and an in-range column).  A warp owns a chunk and
// a lane its row, so every load of the column indices and of the split values is one
// coalesced 128-byte access (the CSR kernel's thread-per-row loads stride by the row
// length); only the gather of x stays irregular (it hits L2: x is one basis column).
// Same arithmetic as k_spmv's double-float rows: TwoProd per nonzero, TwoSum per add.
struct SellArgs {
    const int* len;           // [nchunks] entries per row of the chunk
    const long long* off;     // [nchunks] first entry of the chunk
    const int* col;           // [entries] column indices
    const float* val;         // [2 * entries]: FP32 hi plane, then lo plane
    long long entries;
    long long nchunks;
    long long n;
    const void* x;            // code column (XFMT >= 0) or FP64 vector (XFMT < 0)
    const double* xscale_dev; // decode scale of the code column (may be null: 1)
    float* ydf;               // y as double-float planes hi[ydf_ld], lo[ydf_ld]
    long long ydf_ld;
    double* part;             // [gridDim.x][2] per-block sum of squares (and 0)
    unsigned int* counter;
    DevState* st;             // omega = ||y|| (last block)
    const int* active;        // skip when *active == 0 (may be null)
};

template <int XFMT>
__global__ void __launch_bounds__(THREADS) k_spmv_sell(SellArgs a)
{
    if (a.active && *a.active == 0) return;
    __shared__ double red_s[THREADS / 32], red_m[THREADS / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    constexpr bool XEXACT = XFMT == F32 || XFMT == F16 || XFMT == BF16 || XFMT == E4M3 || XFMT == I16;
    const double xs = a.xscale_dev ? *a.xscale_dev : 1.0;
    const bool xsplit = xs != 1.0;
    float xsh = 1.f, xsl = 0.f;
    if (xsplit) split_f64(xs, xsh, xsl);
    const float* vh = a.val;
    const float* vl = a.val + a.entries;
    float ssS = 0.f, ssC = 0.f;
    auto dfadd = [](float& S, float& C, float pr, float er) {   // (S, C) += pr + er
        const float t = __fadd_rn(S, pr), bb = __fsub_rn(t, S);
        C = __fadd_rn(C, __fadd_rn(__fadd_rn(__fsub_rn(S, __fsub_rn(t, bb)), __fsub_rn(pr, bb)), er));
        S = t;
    };
    for (long long c = (long long)blockIdx.x * (THREADS / 32) + warp; c < a.nchunks;
         c += (long long)gridDim.x * (THREADS / 32)) {
        const int len = a.len[c];
        const long long p0 = a.off[c] + lane;
        float S = 0.f, C = 0.f;
        int k = 0;
        for (; k + 2 <= len; k += 2) {                 // two entries' loads in flight
            const long long p = p0 + 32ll * k, q = p + 32;
            int c0 = a.col[p], c1 = a.col[q];
            float h0 = vh[p], l0 = vl[p], h1 = vh[q], l1 = vl[q];
            if (!col_ok(c0, a.n, a.st)) { c0 = 0; h0 = l0 = 0.f; }
            if (!col_ok(c1, a.n, a.st)) { c1 = 0; h1 = l1 = 0.f; }
            float x0h, x0l, x1h, x1l;
            xval_df<XFMT>(a.x, c0, x0h, x0l);
            xval_df<XFMT>(a.x, c1, x1h, x1l);
            float pr = __fmul_rn(h0, x0h), er = __fmaf_rn(h0, x0h, -pr);
            er = __fmaf_rn(l0, x0h, er);
            if constexpr (!XEXACT) er = __fmaf_rn(h0, x0l, er);
            dfadd(S, C, pr, er);
            pr = __fmul_rn(h1, x1h);
            er = __fmaf_rn(h1, x1h, -pr);
            er = __fmaf_rn(l1, x1h, er);
            if constexpr (!XEXACT) er = __fmaf_rn(h1, x1l, er);
            dfadd(S, C, pr, er);
        }
        if (k < len) {
            const long long p = p0 + 32ll * k;
            int c0 = a.col[p];
            float h0 = vh[p], l0 = vl[p];
            if (!col_ok(c0, a.n, a.st)) { c0 = 0; h0 = l0 = 0.f; }
            float xh, xl;
            xval_df<XFMT>(a.x, c0, xh, xl);
            const float pr = __fmul_rn(h0, xh);
            float er = __fmaf_rn(h0, xh, -pr);
            er = __fmaf_rn(l0, xh, er);
            if constexpr (!XEXACT) er = __fmaf_rn(h0, xl, er);
            dfadd(S, C, pr, er);
        }
        const long long row = c * 32 + lane;
        if (row < a.n) {
            float hi, lo;
            two_sum(S, C, hi, lo);                       // renormalise
            if (xsplit) {                                // integer / power-of-two scales
                const float p = __fmul_rn(hi, xsh);
                float e = __fmaf_rn(hi, xsh, -p);
                e = __fmaf_rn(hi, xsl, e);
                e = __fmaf_rn(lo, xsh, e);
                two_sum(p, e, hi, lo);
            }
            a.ydf[row] = hi;
            a.ydf[a.ydf_ld + row] = lo;
            const float p = __fmul_rn(hi, hi);           // ||y||^2 in double-float
            float e = __fmaf_rn(hi, hi, -p);
            e = __fmaf_rn(__fadd_rn(hi, hi), lo, e);
            dfadd(ssS, ssC, p, e);
        }
    }
    double t, tm;
    block_sum_max(df_to_double(ssS, ssC), 0.0, red_s, red_m, t, tm);
    if (threadIdx.x == 0) {
        a.part[2 * blockIdx.x] = t;
        a.part[2 * blockIdx.x + 1] = 0.0;
    }
    if (last_block(a.counter)) {
        double s2, m2;
        block_reduce_norm_parts(a.part, gridDim.x, s2, m2);
        if (threadIdx.x == 0) a.st->omega = sqrt(s2);
    }
}

// ================================================================ codec test kernels
template <int FMT>
__global__ void k_encode_vec(const double* v, long long n, unsigned char* codes, EncParams ep)
{
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        encode_store<FMT>(codes, i, v[i], ep);
}

template <int FMT>
__global__ void k_decode_vec(const unsigned char* codes, long long n, double scale, double* out)
{
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        out[i] = __dmul_rn(code_value<FMT>(codes, i), scale);
}

}  // namespace cbg
