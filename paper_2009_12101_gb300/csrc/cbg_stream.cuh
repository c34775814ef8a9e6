// cbg_stream.cuh -- the basis dot product h = V^T w (the CGS projection and its re-orthogonalisation, Fig. 1) with the
// compressed basis staged in shared memory by bulk copies (TMA).
//
// One block per SM: sixteen consumer warps and one producer warp.  The work items are
// the (column group, row tile) pairs, numbered group-major (TILE = 8 row groups x 32
// lanes x E rows, E = 16 / bytes per code, so one tile of one column is 4 KiB of codes),
// and a block owns a contiguous range of items, so the blocks' shares differ by at most
// one item (a block may start or end inside a column group).  The producer walks the
// block's items and for each one fills a
// stage of a ring in shared memory with one bulk copy per column (4 KiB each, L2
// evict-first) plus the tile of w as FP32 hi and lo planes; completion is counted in
// bytes on the stage's "full" mbarrier.  Consumer warp w takes row group w % 8 and half
// w / 8 of the stage's columns; its lanes own E consecutive rows, read their 16-byte code
// chunks from shared memory (a warp reads 512 contiguous bytes: no bank conflicts), and
// accumulate in double-float on the packed FP32x2 pipe; each warp releases the stage on
// its "empty" mbarrier.  Loads in flight are bounded by the ring (about 200 KiB per SM),
// not by registers, and the arithmetic never waits on a global load.  Every wait is
// bounded (cbg_tma.cuh): a pipeline that stops making progress records FAULT_TIMEOUT and
// the kernel returns after draining its own copies.
#pragma once
#include "cbg_kernels.cuh"
#include "cbg_tma.cuh"

namespace cbg {

constexpr int TMA_CW = 8;                            // row groups of a tile
constexpr int DOT_CW = 2 * TMA_CW;                   // consumer warps: two per row group
constexpr int DOT_THREADS = (DOT_CW + 1) * 32;       // + one producer warp
constexpr int TMA_SMEM_OPTIN = 232448;               // shared memory per block (227 KiB)
constexpr int TMA_MAX_STAGES = 4;

template <int FMT> struct TmaGeom {
    static constexpr int BS = FmtInfo<FMT>::bytes;
    static constexpr int E = 16 / BS;                // rows per lane (a 16-byte code chunk)
    static constexpr int TILE = TMA_CW * 32 * E;     // rows per tile
    static constexpr int COLB = TILE * BS;           // bytes of one column's tile (4096)
    static constexpr int CG_DOT = E >= 8 ? 8 : 16;   // columns per stage (register accumulators)
    static constexpr int WB = TILE * 8;              // w tile: FP32 hi plane then lo plane
    static constexpr int STAGE_DOT = CG_DOT * COLB + WB;
};

// Dynamic shared memory of the pipelined dot: `stages` ring stages and 2 x stages
// mbarriers.  The ring gets whatever the kernel's static shared memory leaves.
inline int tma_stages(int stage_bytes, int static_bytes)
{
    const int s = (TMA_SMEM_OPTIN - static_bytes - 2 * TMA_MAX_STAGES * 8) / stage_bytes;
    return s < TMA_MAX_STAGES ? s : TMA_MAX_STAGES;
}
inline size_t tma_smem_bytes(int stages, int stage_bytes) { return (size_t)stages * stage_bytes + 2 * (size_t)stages * 8; }

// the block's contiguous range [ib, ie) of nitems work items
__device__ __forceinline__ void block_items(long long nitems, long long& ib, long long& ie)
{
    ib = (long long)blockIdx.x * nitems / gridDim.x;
    ie = ((long long)blockIdx.x + 1) * nitems / gridDim.x;
}

__device__ __forceinline__ void record_fault(DevState* st, int* fault)
{
    if (fault) atomicExch(fault, FAULT_TIMEOUT);
    else if (st) atomicExch(&st->fault, FAULT_TIMEOUT);
}

// Barrier of all blocks of a cooperative launch on one counter word: bits 0..30 count the
// arrivals, bit 31 is the sense, flipped by the last arrival (which also zeroes the
// count), so the word is ready for the next launch as it is left.  Thread 0 of each
// block arrives and waits (bounded: false when the wait gave up); the fences order the
// block's writes before its arrival and the other blocks' writes before its departure.
__device__ __forceinline__ bool grid_barrier(unsigned int* cnt, long long limit)
{
    __shared__ int ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        const unsigned sense = *(volatile unsigned*)cnt & 0x80000000u;
        const unsigned old = atomicAdd(cnt, 1u);
        int good = 1;
        if ((old & 0x7FFFFFFFu) == gridDim.x - 1) {
            atomicExch(cnt, sense ^ 0x80000000u);
        } else {
            const long long t0 = clock64();
            while ((*(volatile unsigned*)cnt & 0x80000000u) == sense) {
                if (clock64() - t0 > limit) {
                    good = 0;
                    break;
                }
                __nanosleep(32);
            }
        }
        __threadfence();
        ok = good;
    }
    __syncthreads();
    return ok != 0;
}

// position in the ring: stage index and the parity of its current use
struct Ring {
    int s = 0;
    unsigned ph = 0;
    __device__ __forceinline__ void next(int stages)
    {
        if (++s == stages) { s = 0; ph ^= 1u; }
    }
};

// E consecutive floats (E a power of two, 4*E-byte aligned) with vector loads
template <int E> __device__ __forceinline__ void load_floats(const float* p, float* out)
{
    if constexpr (E == 2) {
        const float2 v = *reinterpret_cast<const float2*>(p);
        out[0] = v.x;
        out[1] = v.y;
    } else {
#pragma unroll
        for (int e = 0; e < E; e += 4) {
            const float4 v = *reinterpret_cast<const float4*>(p + e);
            out[e] = v.x;
            out[e + 1] = v.y;
            out[e + 2] = v.z;
            out[e + 3] = v.w;
        }
    }
}

// Producer side of the ring: for every work item (group-major), wait until the consumers
// released the stage, announce the bytes, and issue the copies (lane q < nc copies column
// c0 + q; lanes 30 and 31 copy the hi and lo planes of w's tile).  Afterwards wait
// (bounded) until every issued copy has landed, so no copy outlives the block.
template <int COLB>
__device__ __forceinline__ void tma_produce(unsigned char* ring, int stage_bytes, int stages, uint64_t* full,
                                            uint64_t* empty, long long ib, long long ie, long long ntiles, int ncols,
                                            int cg, const unsigned char* V, long long ldb, const float* wsrc,
                                            long long wld, int tile_rows, int* failed, long long limit, bool withhold)
{
    const int lane = threadIdx.x & 31;
    const long long nitems = ie - ib;
    const uint64_t pol = l2_evict_first_policy();
    const unsigned wplane = (unsigned)tile_rows * 4u;
    Ring rg;
    int g = ntiles > 0 ? (int)(ib / ntiles) : 0;
    long long t = ib - (long long)g * ntiles, it = 0;
    for (; it < nitems; it++) {
        const int c0 = g * cg;
        const int nc = ncols - c0 < cg ? ncols - c0 : cg;
        if (it >= stages && !warp_wait(&empty[rg.s], rg.ph ^ 1u, limit)) { *failed = 1; break; }
        unsigned char* st = ring + (size_t)rg.s * stage_bytes;
        if (!(withhold && it == 0)) {
            if (lane == 0) mbar_arrive_expect_tx(&full[rg.s], (unsigned)(nc * COLB) + 2u * wplane);
            __syncwarp();
            if (lane < nc)
                bulk_g2s_hint(st + lane * COLB, V + (long long)(c0 + lane) * ldb + t * COLB, COLB, &full[rg.s], pol);
            if (lane >= 30) {
                const float* src = wsrc + (lane == 31 ? wld : 0) + t * tile_rows;
                bulk_g2s(st + cg * COLB + (lane == 31 ? wplane : 0u), src, wplane, &full[rg.s]);
            }
        }
        __syncwarp();
        rg.next(stages);
        if (++t == ntiles) { t = 0; g++; }
    }
    // drain: walk back over the last min(it, stages) items, the newest use of each stage
    const long long nd = it < stages ? it : stages;
    for (long long j = 0; j < nd; j++) {
        if (--rg.s < 0) { rg.s = stages - 1; rg.ph ^= 1u; }
        if (!warp_wait(&full[rg.s], rg.ph, limit)) { *failed = 1; break; }
    }
}

// ============================================================== h = V^T w  (CGS)
// Consumer warp of the dot: rows r .. r+E-1 of the tile and the CGW = CG/2 columns
// starting at q0 within the stage, as packed pairs.  A missing column (>= nc) holds
// stale codes; its lane of the pair is never read back (only columns < nc are kept).
template <int FMT, bool FULL>
__device__ __forceinline__ void dot_consume(const unsigned char* st, int r, int q0, int nc, float2* S2, float2* C2)
{
    using G = TmaGeom<FMT>;
    constexpr int E = G::E, CG = G::CG_DOT, CGW = CG / 2, BS = G::BS;
    float wh[E], wl[E];
    const float* wt = reinterpret_cast<const float*>(st + CG * G::COLB);
    load_floats<E>(wt + r, wh);
    load_floats<E>(wt + G::TILE + r, wl);
#pragma unroll
    for (int q = 0; q < CGW; q += 2) {
        if (!FULL && q0 + q >= nc) break;
        const uint4 r0 = *reinterpret_cast<const uint4*>(st + (q0 + q) * G::COLB + r * BS);
        const uint4 r1 = *reinterpret_cast<const uint4*>(st + (q0 + q + 1) * G::COLB + r * BS);
        Chunk<FMT> c0h, c1h;
        decode_chunk<FMT>(r0, c0h);
        decode_chunk<FMT>(r1, c1h);
#pragma unroll
        for (int e = 0; e < E; e++) {
            const float2 wh2 = make_float2(wh[e], wh[e]), nwh2 = make_float2(-wh[e], -wh[e]);
            const float2 wl2 = make_float2(wl[e], wl[e]);
            if constexpr (SingleFloat<FMT>::value)
                df2_mac(S2[q / 2], C2[q / 2], make_float2(c0h.vh[e], c1h.vh[e]), wh2, nwh2, wl2);
            else
                df2_mac2(S2[q / 2], C2[q / 2], make_float2(c0h.vh[e], c1h.vh[e]), make_float2(c0h.vl[e], c1h.vl[e]),
                         wh2, nwh2, wl2);
        }
        df2_renorm(S2[q / 2], C2[q / 2]);
    }
}

// barrier among the dot's consumer warps only (the producer never takes part)
__device__ __forceinline__ void consumers_sync()
{
    asm volatile("bar.sync 1, %0;" ::"r"(DOT_CW * 32) : "memory");
}

// DF32 arithmetic; a.wdf (w split into FP32 hi and lo planes) is required.  Sixteen
// consumer warps: warp w takes rows group (w % 8) of every tile and half (w / 8) of every
// stage's columns.  At the end of every column group the consumer warps meet once (a
// hardware barrier) and the group's per-warp sums are added in a fixed order, so the
// block's column totals need only MAXCOLS doubles of shared memory.  A warp whose wait
// timed out stops computing and stops releasing stages but still takes every group
// barrier, so the other warps never wait on it forever.
template <int FMT>
__global__ void __launch_bounds__(DOT_THREADS, 1) k_basis_dot_tma(DotArgs a, int stages, int* fault)
{
    if (a.active && *a.active == 0) return;
    using G = TmaGeom<FMT>;
    constexpr int CG = G::CG_DOT, CGW = CG / 2, E = G::E;
    constexpr int LOW = fold_low<CGW>();
    extern __shared__ __align__(128) unsigned char tma_smem[];
    unsigned char* ring = tma_smem;
    uint64_t* full = reinterpret_cast<uint64_t*>(tma_smem + (size_t)stages * G::STAGE_DOT);
    uint64_t* empty = full + stages;
    __shared__ double red_g[2][TMA_CW][CG];   // per row group sums of the current group (double-buffered)
    __shared__ double red_tot[MAXCOLS];       // the block's column totals
    __shared__ int failed;
    const int ncols = a.ncols_dev ? *a.ncols_dev : a.ncols;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const long long limit = a.wait_limit > 0 ? a.wait_limit : WAIT_LIMIT_CYCLES;
    const long long ntiles = a.nrows / G::TILE;
    const int ngroups = (ncols + CG - 1) / CG;
    long long ib, ie;
    block_items(ntiles * ngroups, ib, ie);

    if (threadIdx.x == 0) {
        failed = 0;
        for (int s = 0; s < stages; s++) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], DOT_CW);
        }
        mbar_init_fence();
    }
    for (int i = threadIdx.x; i < MAXCOLS; i += DOT_THREADS) red_tot[i] = 0.0;
    __syncthreads();

    if (warp == DOT_CW) {
        int f = 0;
        tma_produce<G::COLB>(ring, G::STAGE_DOT, stages, full, empty, ib, ie, ntiles, ncols, CG, a.V, a.ldb, a.wdf,
                             a.nrows, G::TILE, &f, limit, a.withhold != 0);
        if (f) failed = 1;
    } else if (ie > ib) {
        const int rgp = warp % TMA_CW, q0 = (warp / TMA_CW) * CGW;
        const int r = (rgp * 32 + lane) * E;      // first row of this lane within a tile
        bool bad = false;
        Ring rg;
        const int gb = (int)(ib / ntiles), ge = (int)((ie - 1) / ntiles) + 1;   // the block's column groups
        for (int g = gb; g < ge; g++) {
            const int c0 = g * CG;
            const int nc = ncols - c0 < CG ? ncols - c0 : CG;
            // this block's tiles of group g
            const long long tb = ib > (long long)g * ntiles ? ib - (long long)g * ntiles : 0;
            const long long te = ie < (long long)(g + 1) * ntiles ? ie - (long long)g * ntiles : ntiles;
            float2 S2[CGW / 2], C2[CGW / 2];
#pragma unroll
            for (int q = 0; q < CGW / 2; q++) { S2[q] = make_float2(0.f, 0.f); C2[q] = make_float2(0.f, 0.f); }
            for (long long t = tb; t < te; t++) {
                if (!bad && !warp_wait(&full[rg.s], rg.ph, limit)) {
                    bad = true;
                    failed = 1;
                }
                if (!bad) {
                    const unsigned char* st = ring + (size_t)rg.s * G::STAGE_DOT;
                    if (nc == CG) dot_consume<FMT, true>(st, r, q0, nc, S2, C2);
                    else dot_consume<FMT, false>(st, r, q0, nc, S2, C2);
                    __syncwarp();
                    if (lane == 0) mbar_arrive(&empty[rg.s]);
                }
                rg.next(stages);
            }
            float S[CGW], C[CGW];
#pragma unroll
            for (int q = 0; q < CGW / 2; q++) {
                S[2 * q] = S2[q].x;
                S[2 * q + 1] = S2[q].y;
                C[2 * q] = C2[q].x;
                C[2 * q + 1] = C2[q].y;
            }
            const int col = df_warp_fold<CGW>(S, C, lane);
            const double wsum = df_to_double(S[0], C[0]);
            if ((lane & LOW) == 0) red_g[g & 1][rgp][q0 + col] = wsum;
            consumers_sync();
            // red_g[g & 1] is rewritten two groups later, after the next barrier
            const int tid = warp * 32 + lane;
            if (tid < nc) {
                double tot = 0.0;
#pragma unroll
                for (int w = 0; w < TMA_CW; w++) tot += red_g[g & 1][w][tid];
                red_tot[c0 + tid] = tot;
            }
        }
    }
    __syncthreads();
    if (failed && threadIdx.x == 0) record_fault(nullptr, fault);
    for (int col = threadIdx.x; col < ncols; col += DOT_THREADS) a.part[(long long)blockIdx.x * MAXCOLS + col] = red_tot[col];
    // Grid barrier (the kernel is launched cooperatively: every block is resident), then
    // block b adds the partials of the columns b, b + gridDim.x, ...: one load per thread
    // and column, one warp shuffle tree per warp, then one over the warps' sums.  The
    // cross-block sum is spread over all SMs instead of one last block, whose FP64 pipe
    // (a few FP64 operations per clock per SM on GB300) and serial L2 round trips would
    // otherwise add tens of microseconds to a launch.
    if (!grid_barrier(a.counter, limit)) {
        if (threadIdx.x == 0) record_fault(nullptr, fault);
        return;
    }
    __shared__ double wsum_sh[DOT_CW + 1][4];
    const int nb = gridDim.x;
    for (int c0 = blockIdx.x; c0 < ncols; c0 += 4 * nb) {
        double v[4] = {0.0, 0.0, 0.0, 0.0};
        for (int t = threadIdx.x; t < nb; t += DOT_THREADS) {   // a thread adds blocks t, t + 544, ...
            double q[4];
#pragma unroll
            for (int k = 0; k < 4; k++) {
                const int col = c0 + k * nb;
                q[k] = col < ncols ? __ldcg(a.part + (long long)t * MAXCOLS + col) : 0.0;
            }
#pragma unroll
            for (int k = 0; k < 4; k++) v[k] += q[k];
        }
#pragma unroll
        for (int k = 0; k < 4; k++) v[k] = warp_sum(v[k]);
        if (lane == 0)
#pragma unroll
            for (int k = 0; k < 4; k++) wsum_sh[warp][k] = v[k];
        __syncthreads();
        if (warp == 0) {
            // the 17 warps' sums of the four columns at once: lane l takes column l / 8 and
            // warps l % 8, l % 8 + 8, l % 8 + 16 (in that order), then a three-level tree
            // within each group of eight lanes
            const int k = lane >> 3, w0 = lane & 7;
            double sum = 0.0;
#pragma unroll
            for (int w = w0; w < DOT_CW + 1; w += 8) sum += wsum_sh[w][k];
#pragma unroll
            for (int o = 4; o > 0; o >>= 1) sum += __shfl_xor_sync(0xFFFFFFFFu, sum, o);
            const int col = c0 + k * nb;
            if (w0 == 0 && col < ncols) a.out[col] = sum * a.scales[col];
        }
        __syncthreads();
    }
}

}  // namespace cbg
