// cbg_batched.cuh -- batched GMRES(m): many independent systems in one persistent launch.
//
// Each system runs the same restarted Arnoldi process as the single-system path (Fig. 1
// with the explicit-residual recheck of Section 5.2), entirely on the device.  The
// launch uses thread-block clusters.  A cluster takes systems from a device work queue
// ordered by decreasing size.  Systems with at least `split_rows` rows are solved by the
// whole cluster (rows split across its blocks; sums through distributed shared memory
// and the hardware cluster barrier); once the queue reaches the small systems, every
// block takes its own systems and runs alone.  No block ever spins on a flag: all waits
// are __syncthreads or cluster barriers, which the hardware guarantees to complete.
//
// Per block, the block's rows of w live in shared memory as double-float pairs; only
// the compressed basis, x and b are in HBM.
#pragma once
#include <cooperative_groups.h>

#include "cbg_device.cuh"

namespace cbg {

namespace cgx = cooperative_groups;

constexpr int BT_THREADS = 256;
constexpr int BT_MAXM = 64;          // largest restart length of the batched kernel
constexpr int BT_OK = 0, BT_NOT_CONVERGED = 1, BT_NONFINITE = -2;   // cbgmres.h status values

struct BatchSys {
    int n;                  // rows
    int ld;                 // padded rows of a basis column (multiple of 64)
    long long rp_off;       // offset of the system's n+1 row pointers
    long long nz_off;       // offset of its nonzeros (column indices are local)
    long long vec_off;      // offset of its b / x / dinv entries
    long long v_off;        // byte offset of its basis
    double pscale;          // 2^s normalising its per-step operator (largest |value| in [1, 2))
    double hscale;          // 2^-s: Hessenberg columns back to the unscaled operator
};

struct BatchOut {
    long long iters;
    long long restarts;
    double relres;
    int status;
    int pad0;
};

struct BatchArgs {
    const BatchSys* sys;
    const int* order;       // queue order (decreasing n)
    int nsys;
    int m;
    const int* rowptr;
    const int* col;
    const double* valp;     // A D^{-1} (Jacobi) or A
    const double* val;      // A
    const double* dinv;     // D^{-1} or null
    const float* valpdf;    // valp times each system's pscale as FP32 hi [nnz_all] then lo
                            // [nnz_all] planes for the per-step SpMV in double-float, or null
                            // (FP64 products)
    long long nnz_all;
    double* const* io;      // io[0] = b (packed), io[1] = x (packed); device table
    unsigned char* V;
    BatchOut* out;
    unsigned int* queue;    // work-queue head (zeroed before every launch)
    double tol;
    long long maxit;
    double eps_bd;
    int split_rows;
    int max_rows_block;     // capacity of the shared-memory w (rows)
    int spmv_lanes;         // SpMV schedule: 1 = a thread per row (4 rows in flight), or 2, 4, 8
                            // lanes per row (the lanes split the row's nonzeros)
};

// shared-memory layout of one block (dynamic)
struct BtSmem {
    double H[(BT_MAXM + 1) * BT_MAXM];
    double g[BT_MAXM + 1], cs[BT_MAXM], sn[BT_MAXM], y[BT_MAXM + 1];
    double h[BT_MAXM + 1], u[BT_MAXM + 1], scale[BT_MAXM + 1];
    double red[BT_MAXM + 4];           // this block's partial sums (read by the cluster)
    double tot[BT_MAXM + 4];           // team totals
    double wred[BT_THREADS / 32][BT_MAXM + 4];
    int sys_idx;
    int stop;
    float2 ws[1];                      // w rows of this block (max_rows_block + 16 entries)
};

template <bool CLUSTER> struct Team {
    int rank, size;
    __device__ __forceinline__ void sync() const
    {
        if constexpr (CLUSTER) {
            __threadfence();
            cgx::this_cluster().sync();
        } else {
            __syncthreads();
        }
    }
    // tot[i] = sum over the team's blocks of red[i], i < k, in block order (identical in
    // every block).
    __device__ __forceinline__ void reduce(BtSmem* sm, int k) const
    {
        if constexpr (CLUSTER) {
            cgx::cluster_group cl = cgx::this_cluster();
            cl.sync();
            for (int i = threadIdx.x; i < k; i += BT_THREADS) {
                double t = 0.0;
                for (int r = 0; r < size; r++) t += cl.map_shared_rank(sm->red, r)[i];
                sm->tot[i] = t;
            }
            cl.sync();
        } else {
            __syncthreads();
            for (int i = threadIdx.x; i < k; i += BT_THREADS) sm->tot[i] = sm->red[i];
            __syncthreads();
        }
    }
};

// block-wide sum of per-thread values v[0..k) into sm->red[0..k) (fixed order)
template <int K>
__device__ __forceinline__ void block_sum(BtSmem* sm, const double (&v)[K], int k, int red_off)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int i = 0; i < K; i++) {
        if (i >= k) break;
        double s = warp_sum(v[i]);
        if (lane == 0) sm->wred[warp][i] = s;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < k; i += BT_THREADS) {
        double s = 0.0;
        for (int w = 0; w < BT_THREADS / 32; w++) s += sm->wred[w][i];
        sm->red[red_off + i] = s;
    }
    __syncthreads();
}

template <int FMT> struct BatchedSolver {
    static constexpr int BS = FmtInfo<FMT>::bytes;
    static constexpr int E = 16 / BS;

    // ------------------------------------------------------------------ block kernels
    // w (own rows) = A_pc x  with x given by codes (column `col`, scaled) or FP64 array;
    // ws <- DF(w).  Returns the thread's sum of w^2.
    template <bool CODES>
    static __device__ double spmv(const BatchArgs& a, const BatchSys& s, BtSmem* sm, int r0, int r1,
                                  const void* x, double xscale, const double* vals, bool residual)
    {
        const int* rp = a.rowptr + s.rp_off;
        const int* ci = a.col + s.nz_off;
        const double* va = vals + s.nz_off;
        const double* bb = a.io[0] + s.vec_off;
        double ss = 0.0;
        constexpr int RW = 4;                              // rows per thread in flight
        for (int rb = r0 + threadIdx.x; rb < r1; rb += RW * BT_THREADS) {
            double t[RW];
            int p0[RW], p1[RW];
#pragma unroll
            for (int q = 0; q < RW; q++) {
                const int r = rb + q * BT_THREADS;
                t[q] = 0.0;
                p0[q] = r < r1 ? rp[r] : 0;
                p1[q] = r < r1 ? rp[r + 1] : 0;
            }
            int len = 0;
#pragma unroll
            for (int q = 0; q < RW; q++) len = max(len, p1[q] - p0[q]);
            for (int i = 0; i < len; i++) {
#pragma unroll
                for (int q = 0; q < RW; q++) {
                    const int p = p0[q] + i;
                    if (p < p1[q]) {
                        double xv;
                        if constexpr (CODES) xv = code_value<FMT>(x, ci[p]);
                        else xv = reinterpret_cast<const double*>(x)[ci[p]];
                        t[q] = __fma_rn(va[p], xv, t[q]);
                    }
                }
            }
#pragma unroll
            for (int q = 0; q < RW; q++) {
                const int r = rb + q * BT_THREADS;
                if (r < r1) {
                    double v = t[q];
                    if constexpr (CODES) v = __dmul_rn(v, xscale);
                    if (residual) v = __dsub_rn(bb[r], v);
                    float hi, lo;
                    split_f64(v, hi, lo);
                    sm->ws[r - r0] = make_float2(hi, lo);
                    ss = __fma_rn(v, v, ss);
                }
            }
        }
        return ss;
    }

    // The per-step w = A_pc v_j in double-float: every product val * code is formed as an
    // FP32 pair (TwoProd on the split values; exact for single-float codes up to the
    // rounding of the lo term) and summed with TwoSum; w goes to ws as its renormalised
    // pair and the sum of w^2 is accumulated in double-float, so no FP64 operation runs
    // per nonzero or per row (GB300's FP64 pipe is ~70x narrower than its FP32 pipe).
    // The planes hold the normalised operator 2^s A_pc.
    static __device__ double spmv_df(const BatchArgs& a, const BatchSys& s, BtSmem* sm, int r0, int r1,
                                     const void* x, double xscale)
    {
        const int* rp = a.rowptr + s.rp_off;
        const int* ci = a.col + s.nz_off;
        const float* vh = a.valpdf + s.nz_off;
        const float* vl = a.valpdf + a.nnz_all + s.nz_off;
        const bool xsplit = xscale != 1.0;                 // unit scale (float formats): no product
        float xsh = 1.f, xsl = 0.f;
        if (xsplit) split_f64(xscale, xsh, xsl);
        float ssS = 0.f, ssC = 0.f;
        constexpr int RW = 4;                              // rows per thread in flight
        for (int rb = r0 + threadIdx.x; rb < r1; rb += RW * BT_THREADS) {
            float S[RW], C[RW];
            int p0[RW], p1[RW];
#pragma unroll
            for (int q = 0; q < RW; q++) {
                const int r = rb + q * BT_THREADS;
                S[q] = 0.f;
                C[q] = 0.f;
                p0[q] = r < r1 ? rp[r] : 0;
                p1[q] = r < r1 ? rp[r + 1] : 0;
            }
            int len = 0;
#pragma unroll
            for (int q = 0; q < RW; q++) len = max(len, p1[q] - p0[q]);
            for (int i = 0; i < len; i++) {
#pragma unroll
                for (int q = 0; q < RW; q++) {
                    const int p = p0[q] + i;
                    if (p < p1[q]) {
                        float xh, xl;
                        xval_df<FMT>(x, ci[p], xh, xl);
                        if constexpr (SingleFloat<FMT>::value) df_mac(S[q], C[q], xh, vh[p], vl[p]);
                        else df_mac2(S[q], C[q], xh, xl, vh[p], vl[p]);
                    }
                }
            }
#pragma unroll
            for (int q = 0; q < RW; q++) {
                const int r = rb + q * BT_THREADS;
                if (r < r1) {
                    float hi, lo;
                    two_sum(S[q], C[q], hi, lo);             // renormalise
                    if (xsplit) {                            // (hi + lo) * (xsh + xsl)
                        const float p = __fmul_rn(hi, xsh);
                        float e = __fmaf_rn(hi, xsh, -p);
                        e = __fmaf_rn(hi, xsl, e);
                        e = __fmaf_rn(lo, xsh, e);
                        two_sum(p, e, hi, lo);
                    }
                    sm->ws[r - r0] = make_float2(hi, lo);
                    // w^2 = hi^2 + 2 hi lo to double-float accuracy
                    const float p = __fmul_rn(hi, hi);
                    float e = __fmaf_rn(hi, hi, -p);
                    e = __fmaf_rn(__fadd_rn(hi, hi), lo, e);
                    float t, te;
                    two_sum(ssS, p, t, te);
                    ssC = __fadd_rn(ssC, __fadd_rn(te, e));
                    ssS = t;
                }
            }
        }
        return df_to_double(ssS, ssC);
    }

    // The SpMVs above with L = a.spmv_lanes lanes per row (L = 2, 4, 8): the lanes of a
    // group take every L-th nonzero of the row and their partial sums meet in shuffles.
    // Groups walk the block's rows in warp-uniform passes, so every shuffle has the whole
    // warp.  Same results up to the order of each row's sum.
    template <bool CODES>
    static __device__ double spmv_lanes(const BatchArgs& a, const BatchSys& s, BtSmem* sm, int r0, int r1,
                                        const void* x, double xscale, const double* vals, bool residual)
    {
        const int* rp = a.rowptr + s.rp_off;
        const int* ci = a.col + s.nz_off;
        const double* va = vals + s.nz_off;
        const double* bb = a.io[0] + s.vec_off;
        const int L = a.spmv_lanes, lg = threadIdx.x & (L - 1), gpw = 32 / L;
        const int gw = (threadIdx.x & 31) / L, warp = threadIdx.x >> 5;
        double ss = 0.0;
        for (int base = r0 + warp * gpw; base < r1; base += (BT_THREADS / 32) * gpw) {
            const int r = base + gw;
            const bool valid = r < r1;
            double t = 0.0;
            if (valid) {
                const int p1 = rp[r + 1];
                for (int p = rp[r] + lg; p < p1; p += L) {
                    double xv;
                    if constexpr (CODES) xv = code_value<FMT>(x, ci[p]);
                    else xv = reinterpret_cast<const double*>(x)[ci[p]];
                    t = __fma_rn(va[p], xv, t);
                }
            }
            for (int o = L >> 1; o > 0; o >>= 1) t = __dadd_rn(t, __shfl_xor_sync(0xffffffffu, t, o));
            if (valid && lg == 0) {
                double v = t;
                if constexpr (CODES) v = __dmul_rn(v, xscale);
                if (residual) v = __dsub_rn(bb[r], v);
                float hi, lo;
                split_f64(v, hi, lo);
                sm->ws[r - r0] = make_float2(hi, lo);
                ss = __fma_rn(v, v, ss);
            }
        }
        return ss;
    }

    static __device__ double spmv_df_lanes(const BatchArgs& a, const BatchSys& s, BtSmem* sm, int r0, int r1,
                                           const void* x, double xscale)
    {
        const int* rp = a.rowptr + s.rp_off;
        const int* ci = a.col + s.nz_off;
        const float* vh = a.valpdf + s.nz_off;
        const float* vl = a.valpdf + a.nnz_all + s.nz_off;
        const bool xsplit = xscale != 1.0;
        float xsh = 1.f, xsl = 0.f;
        if (xsplit) split_f64(xscale, xsh, xsl);
        const int L = a.spmv_lanes, lg = threadIdx.x & (L - 1), gpw = 32 / L;
        const int gw = (threadIdx.x & 31) / L, warp = threadIdx.x >> 5;
        float ssS = 0.f, ssC = 0.f;
        for (int base = r0 + warp * gpw; base < r1; base += (BT_THREADS / 32) * gpw) {
            const int r = base + gw;
            const bool valid = r < r1;
            float S = 0.f, C = 0.f;
            if (valid) {
                const int p1 = rp[r + 1];
                for (int p = rp[r] + lg; p < p1; p += L) {
                    float xh, xl;
                    xval_df<FMT>(x, ci[p], xh, xl);
                    if constexpr (SingleFloat<FMT>::value) df_mac(S, C, xh, vh[p], vl[p]);
                    else df_mac2(S, C, xh, xl, vh[p], vl[p]);
                }
            }
            for (int o = L >> 1; o > 0; o >>= 1) {
                const float S2 = __shfl_xor_sync(0xffffffffu, S, o), C2 = __shfl_xor_sync(0xffffffffu, C, o);
                df_add(S, C, S2, C2);
            }
            if (valid && lg == 0) {
                float hi, lo;
                two_sum(S, C, hi, lo);
                if (xsplit) {
                    const float p = __fmul_rn(hi, xsh);
                    float e = __fmaf_rn(hi, xsh, -p);
                    e = __fmaf_rn(hi, xsl, e);
                    e = __fmaf_rn(lo, xsh, e);
                    two_sum(p, e, hi, lo);
                }
                sm->ws[r - r0] = make_float2(hi, lo);
                const float p = __fmul_rn(hi, hi);
                float e = __fmaf_rn(hi, hi, -p);
                e = __fmaf_rn(__fadd_rn(hi, hi), lo, e);
                float t, te;
                two_sum(ssS, p, t, te);
                ssC = __fadd_rn(ssC, __fadd_rn(te, e));
                ssS = t;
            }
        }
        return df_to_double(ssS, ssC);
    }

    // partial h_k = sum over own rows of dec(V_k) w, k < ncols, into sm->red[0..ncols)
    // (scale applied); one warp per column, lanes walk the rows in 16-byte chunks.
    static __device__ void dot(const BatchArgs& a, const BatchSys& s, BtSmem* sm, int r0, int r1, int ncols)
    {
        const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
        const unsigned char* Vs = a.V + s.v_off;
        const int nloc = r1 - r0;
        constexpr int U = 8;                               // 16-byte loads in flight per lane
        for (int k = warp; k < ncols; k += BT_THREADS / 32) {
            const unsigned char* cp = Vs + ((long long)k * s.ld + r0) * BS;
            float S = 0.f, C = 0.f;
            for (int b0 = lane * E; b0 < nloc; b0 += U * 32 * E) {
                uint4 raw[U];
#pragma unroll
                for (int q = 0; q < U; q++) {
                    const int e0 = b0 + q * 32 * E;
                    raw[q] = e0 < nloc ? ldg_stream(cp + (long long)e0 * BS) : make_uint4(0u, 0u, 0u, 0u);
                }
#pragma unroll
                for (int q = 0; q < U; q++) {
                    const int e0 = b0 + q * 32 * E;
                    if (e0 >= nloc) break;
                    Chunk<FMT> ch;
                    decode_chunk<FMT>(raw[q], ch);
#pragma unroll
                    for (int e = 0; e < E; e++) {
                        const float2 wv = sm->ws[e0 + e];      // zero beyond nloc
                        if constexpr (SingleFloat<FMT>::value) df_mac(S, C, ch.vh[e], wv.x, wv.y);
                        else df_mac2(S, C, ch.vh[e], ch.vl[e], wv.x, wv.y);
                    }
                    df_renorm(S, C);
                }
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                const float oS = __shfl_xor_sync(0xFFFFFFFFu, S, o);
                const float oC = __shfl_xor_sync(0xFFFFFFFFu, C, o);
                df_add(S, C, oS, oC);
            }
            if (lane == 0) sm->red[k] = __dmul_rn(df_to_double(S, C), sm->scale[k]);
        }
        __syncthreads();
    }

    // ws -= V coef over own rows; with NORMS, also the thread's sum of squares and max |w|
    // of the result (FP64 from the DF value; only the last pass of a step needs them).
    template <bool NORMS>
    static __device__ void axpy(const BatchArgs& a, const BatchSys& s, BtSmem* sm, int r0, int r1, int ncols,
                                const double* coef, double& ss, double& mx)
    {
        __shared__ float2 cdf[BT_MAXM + 1];
        for (int k = threadIdx.x; k < ncols; k += BT_THREADS) {
            float hi, lo;
            split_f64(-coef[k] * sm->scale[k], hi, lo);
            cdf[k] = make_float2(hi, lo);
        }
        __syncthreads();
        const unsigned char* Vs = a.V + s.v_off;
        const int nloc = r1 - r0;
        ss = 0.0;
        mx = 0.0;
        for (int e0 = threadIdx.x * E; e0 < nloc; e0 += BT_THREADS * E) {
            float S[E], C[E];
#pragma unroll
            for (int e = 0; e < E; e++) { S[e] = sm->ws[e0 + e].x; C[e] = sm->ws[e0 + e].y; }
            const unsigned char* base = Vs + ((long long)r0 + e0) * BS;
            constexpr int U = E <= 8 ? 8 : 4;                // columns in flight per thread
            for (int k0 = 0; k0 < ncols; k0 += U) {
                uint4 raw[U];
#pragma unroll
                for (int q = 0; q < U; q++)
                    raw[q] = k0 + q < ncols ? ldg_stream(base + (long long)(k0 + q) * s.ld * BS)
                                            : make_uint4(0u, 0u, 0u, 0u);
#pragma unroll
                for (int q = 0; q < U; q++) {
                    if (k0 + q >= ncols) break;
                    Chunk<FMT> ch;
                    decode_chunk<FMT>(raw[q], ch);
                    const float2 c = cdf[k0 + q];
#pragma unroll
                    for (int e = 0; e < E; e++) {
                        if constexpr (SingleFloat<FMT>::value) df_mac(S[e], C[e], ch.vh[e], c.x, c.y);
                        else df_mac2(S[e], C[e], ch.vh[e], ch.vl[e], c.x, c.y);
                    }
                    if ((q & 3) == 3) {
#pragma unroll
                        for (int e = 0; e < E; e++) df_renorm(S[e], C[e]);
                    }
                }
            }
#pragma unroll
            for (int e = 0; e < E; e++) {
                if (e0 + e < nloc) {
                    df_renorm(S[e], C[e]);
                    sm->ws[e0 + e] = make_float2(S[e], C[e]);
                    if constexpr (NORMS) {
                        const double d = df_to_double(S[e], C[e]);
                        ss = __fma_rn(d, d, ss);
                        // max |d| through the bit pattern (integer compare of non-negative doubles)
                        const long long ab = __double_as_longlong(d) & 0x7FFFFFFFFFFFFFFFll;
                        mx = ab > __double_as_longlong(mx) ? __longlong_as_double(ab) : mx;
                    }
                }
            }
        }
        __syncthreads();
    }

    // store v = w * inv (own rows) into basis column `col`
    static __device__ void encode(const BatchArgs& a, const BatchSys& s, BtSmem* sm, int r0, int r1, int col,
                                  double inv, const EncParams& ep)
    {
        unsigned char* dst = a.V + s.v_off + (long long)col * s.ld * BS;
        for (int r = r0 + threadIdx.x; r < r1; r += BT_THREADS) {
            const float2 wv = sm->ws[r - r0];
            encode_store<FMT>(dst, r, __dmul_rn(df_to_double(wv.x, wv.y), inv), ep);
        }
    }

    // --------------------------------------------------------------------- one system
    template <bool CLUSTER>
    static __device__ void solve(const BatchArgs& a, int si, BtSmem* sm, const Team<CLUSTER>& team)
    {
        const BatchSys s = a.sys[si];
        const int m = a.m;
        const int chunk = ((s.n + team.size - 1) / team.size + 15) / 16 * 16;
        const int r0 = min(s.n, team.rank * chunk);
        const int r1 = min(s.n, r0 + chunk);
        const int nloc = r1 - r0;
        // zero the w rows (and the 16-entry tail read by the chunked loops)
        for (int i = threadIdx.x; i < nloc + 16; i += BT_THREADS) sm->ws[i] = make_float2(0.f, 0.f);
        double* x = a.io[1] + s.vec_off;
        const double* dinv = a.dinv ? a.dinv + s.vec_off : nullptr;

        // ||b||
        {
            double v[1] = {0.0};
            for (int r = r0 + threadIdx.x; r < r1; r += BT_THREADS) {
                const double bv = a.io[0][s.vec_off + r];
                v[0] = __fma_rn(bv, bv, v[0]);
            }
            block_sum<1>(sm, v, 1, 0);
            team.reduce(sm, 1);
        }
        const double bnorm = sqrt(sm->tot[0]);
        long long iters = 0, cycles = 0;
        int status = BT_NOT_CONVERGED;
        double beta = 0.0;
        if (bnorm == 0.0) {
            for (int r = r0 + threadIdx.x; r < r1; r += BT_THREADS) x[r] = 0.0;
            status = 0;
        } else {
            const double target = a.tol * bnorm;
            for (;;) {
                // residual r = b - A x into ws; beta, ||r||_inf
                team.sync();                                   // x of all blocks visible
                double v[2];
                v[0] = a.spmv_lanes > 1 ? spmv_lanes<false>(a, s, sm, r0, r1, x, 1.0, a.val, true)
                                        : spmv<false>(a, s, sm, r0, r1, x, 1.0, a.val, true);
                v[1] = 0.0;
                double mxl = 0.0;
                for (int r = r0 + threadIdx.x; r < r1; r += BT_THREADS) {
                    const float2 wv = sm->ws[r - r0];
                    mxl = fmax(mxl, fabs(df_to_double(wv.x, wv.y)));
                }
                {
                    __syncthreads();
                    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
                    double s2 = warp_sum(v[0]), m2 = warp_max(mxl);
                    if (lane == 0) { sm->wred[warp][0] = s2; sm->wred[warp][1] = m2; }
                    __syncthreads();
                    if (threadIdx.x == 0) {
                        double t = 0.0, mm = 0.0;
                        for (int w = 0; w < BT_THREADS / 32; w++) { t += sm->wred[w][0]; mm = fmax(mm, sm->wred[w][1]); }
                        sm->red[0] = t;
                        sm->red[1] = mm;
                    }
                }
                // the max is combined through the same fixed-order path (sum of block maxima
                // is not needed: take the max over blocks explicitly)
                team.reduce(sm, 1);
                beta = sqrt(sm->tot[0]);
                double rinf = sm->red[1];
                if constexpr (CLUSTER) {
                    cgx::cluster_group cl = cgx::this_cluster();
                    for (int r = 0; r < team.size; r++) rinf = fmax(rinf, cl.map_shared_rank(sm->red, r)[1]);
                    cl.sync();
                }
                if (!(beta > target)) { status = isfinite(beta) ? 0 : BT_NONFINITE; break; }
                if (iters >= a.maxit) { status = BT_NOT_CONVERGED; break; }
                cycles++;
                const long long left = a.maxit - iters;
                const int kcap = (int)(left < m ? left : m);
                // v_1 = r / beta
                {
                    const double inv = 1.0 / beta;
                    const EncParams ep = enc_params(FMT, __dmul_rn(rinf, inv));
                    if (threadIdx.x == 0) sm->scale[0] = ep.scale;
                    encode(a, s, sm, r0, r1, 0, inv, ep);
                }
                for (int i = threadIdx.x; i <= m; i += BT_THREADS) { sm->g[i] = 0.0; sm->y[i] = 0.0; }
                if (threadIdx.x == 0) sm->g[0] = beta;
                int k = 0;
                for (int j = 0; j < kcap; j++) {
                    team.sync();                               // column j of all blocks visible
                    // w = 2^s A D^{-1} v_j (the normalised operator; Jacobi folded into the
                    // values), omega = ||w||.  Double-float products unless the planes are
                    // absent; f64 codes keep FP64 products, which measured faster than
                    // splitting every gathered code.
                    double om[1];
                    const unsigned char* vj = a.V + s.v_off + (long long)j * s.ld * BS;
                    const double xs = __dmul_rn(sm->scale[j], s.pscale);
                    if (FMT != F64 && a.valpdf)                  // planes hold 2^s A_pc
                        om[0] = a.spmv_lanes > 1 ? spmv_df_lanes(a, s, sm, r0, r1, vj, sm->scale[j])
                                                 : spmv_df(a, s, sm, r0, r1, vj, sm->scale[j]);
                    else
                        om[0] = a.spmv_lanes > 1 ? spmv_lanes<true>(a, s, sm, r0, r1, vj, xs, a.valp, false)
                                                 : spmv<true>(a, s, sm, r0, r1, vj, xs, a.valp, false);
                    __syncthreads();
                    block_sum<1>(sm, om, 1, j + 1);              // red[j+1] = omega^2 partial
                    dot(a, s, sm, r0, r1, j + 1);                // red[0..j]
                    team.reduce(sm, j + 2);
                    const double omega = sqrt(sm->tot[j + 1]);
                    for (int i = threadIdx.x; i <= j; i += BT_THREADS) sm->h[i] = sm->tot[i];
                    __syncthreads();
                    double ss, mx;
                    axpy<false>(a, s, sm, r0, r1, j + 1, sm->h, ss, mx);   // (norms of w1 unused)
                    dot(a, s, sm, r0, r1, j + 1);
                    team.reduce(sm, j + 1);
                    for (int i = threadIdx.x; i <= j; i += BT_THREADS) sm->u[i] = sm->tot[i];
                    __syncthreads();
                    axpy<true>(a, s, sm, r0, r1, j + 1, sm->u, ss, mx);
                    double nv[1] = {ss};
                    block_sum<1>(sm, nv, 1, 0);
                    {   // block max of |w|
                        const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
                        double m2 = warp_max(mx);
                        if (lane == 0) sm->wred[warp][1] = m2;
                        __syncthreads();
                        if (threadIdx.x == 0) {
                            double mm = 0.0;
                            for (int w = 0; w < BT_THREADS / 32; w++) mm = fmax(mm, sm->wred[w][1]);
                            sm->red[1] = mm;
                        }
                    }
                    team.reduce(sm, 1);
                    const double hn = sqrt(sm->tot[0]);
                    double wmax = sm->red[1];
                    if constexpr (CLUSTER) {
                        cgx::cluster_group cl = cgx::this_cluster();
                        for (int r = 0; r < team.size; r++) wmax = fmax(wmax, cl.map_shared_rank(sm->red, r)[1]);
                        cl.sync();
                    }
                    // Hessenberg column (scaled back from the normalised operator, exactly),
                    // Givens rotations, stopping tests (identical in every block)
                    if (threadIdx.x == 0) {
                        double* Hc = sm->H + j * (m + 1);
                        for (int i = 0; i <= j; i++) Hc[i] = __dmul_rn(__dadd_rn(sm->h[i], sm->u[i]), s.hscale);
                        const double hnt = __dmul_rn(hn, s.hscale);
                        Hc[j + 1] = hnt;
                        double r0v = Hc[0];
                        for (int i = 0; i < j; i++) {
                            const double c = sm->cs[i], sn = sm->sn[i], r1v = Hc[i + 1];
                            Hc[i] = __dadd_rn(__dmul_rn(c, r0v), __dmul_rn(sn, r1v));
                            r0v = __dadd_rn(__dmul_rn(-sn, r0v), __dmul_rn(c, r1v));
                        }
                        const double rr = hypot(r0v, hnt);
                        double c = 1.0, sn = 0.0;
                        if (rr != 0.0) { c = r0v / rr; sn = hnt / rr; }
                        sm->cs[j] = c;
                        sm->sn[j] = sn;
                        Hc[j] = rr;
                        Hc[j + 1] = 0.0;
                        const double gj = sm->g[j];
                        sm->g[j + 1] = __dmul_rn(-sn, gj);
                        sm->g[j] = __dmul_rn(c, gj);
                        const double est = fabs(sm->g[j + 1]);
                        int stop = 0;
                        if (!isfinite(hnt) || !isfinite(omega) || !isfinite(est)) stop = 3;
                        else if (!(hn > a.eps_bd * omega)) stop = 2;        // both of the scaled operator
                        else if (est <= target) stop = 1;
                        else if (j + 1 >= kcap) stop = 4;
                        sm->stop = stop;
                    }
                    __syncthreads();
                    iters++;
                    k = j + 1;
                    if (sm->stop) break;
                    const double inv = 1.0 / hn;
                    const EncParams ep = enc_params(FMT, __dmul_rn(wmax, inv));
                    if (threadIdx.x == 0) sm->scale[j + 1] = ep.scale;
                    encode(a, s, sm, r0, r1, j + 1, inv, ep);
                }
                if (sm->stop == 3) { status = BT_NONFINITE; break; }
                // y = R^{-1} g (Hessenberg columns hold R after the rotations)
                if (threadIdx.x == 0) {
                    for (int i = k - 1; i >= 0; i--) {
                        double t = sm->g[i];
                        for (int c2 = i + 1; c2 < k; c2++) t = __dsub_rn(t, __dmul_rn(sm->H[i + c2 * (m + 1)], sm->y[c2]));
                        sm->y[i] = t / sm->H[i + i * (m + 1)];
                    }
                }
                __syncthreads();
                // x += D^{-1} V y over own rows
                {
                    const unsigned char* Vs = a.V + s.v_off;
                    for (int r = r0 + threadIdx.x; r < r1; r += BT_THREADS) {
                        double t = 0.0;
                        for (int c2 = 0; c2 < k; c2++)
                            t = __fma_rn(__dmul_rn(code_value<FMT>(Vs + (long long)c2 * s.ld * BS, r), sm->scale[c2]),
                                         sm->y[c2], t);
                        if (dinv) t = __dmul_rn(dinv[r], t);
                        x[r] = __dadd_rn(x[r], t);
                    }
                }
            }
        }
        if (team.rank == 0 && threadIdx.x == 0) {
            a.out[si].iters = iters;
            a.out[si].restarts = cycles;
            a.out[si].relres = bnorm > 0.0 ? beta / bnorm : 0.0;
            a.out[si].status = status;
        }
        team.sync();
    }
};

template <int FMT>
__global__ void __launch_bounds__(BT_THREADS, 2) k_batched(BatchArgs a)
{
    extern __shared__ __align__(16) unsigned char bt_smem_raw[];
    BtSmem* sm = reinterpret_cast<BtSmem*>(bt_smem_raw);
    cgx::cluster_group cl = cgx::this_cluster();
    const int crank = (int)cl.block_rank(), csize = (int)cl.num_blocks();
    int mine = -1;
    // cluster phase: large systems, one cluster each
    for (;;) {
        if (crank == 0 && threadIdx.x == 0) sm->sys_idx = (int)atomicAdd(a.queue, 1u);
        cl.sync();
        const int idx = *cl.map_shared_rank(&sm->sys_idx, 0);
        cl.sync();
        if (idx >= a.nsys) return;                           // every block of the cluster leaves together
        const int si = a.order[idx];
        if (csize > 1 && a.sys[si].n >= a.split_rows) {
            Team<true> t{crank, csize};
            BatchedSolver<FMT>::template solve<true>(a, si, sm, t);
            continue;
        }
        mine = crank == 0 ? si : -1;                         // small systems from here on
        break;
    }
    // block phase: small systems, one block each (no cluster-wide operation any more)
    for (;;) {
        if (mine < 0) {
            __syncthreads();
            if (threadIdx.x == 0) sm->sys_idx = (int)atomicAdd(a.queue, 1u);
            __syncthreads();
            const int idx = sm->sys_idx;
            if (idx >= a.nsys) return;
            mine = a.order[idx];
        }
        Team<false> t{0, 1};
        BatchedSolver<FMT>::template solve<false>(a, mine, sm, t);
        mine = -1;
    }
}

}  // namespace cbg
