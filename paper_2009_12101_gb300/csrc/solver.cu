// solver.cu -- host driver of the restarted Arnoldi process and the C ABI (cbgmres.h).
//
// One restart cycle (Fig. 1):
//   residual kernel     r = b - A x, beta = ||r||, ||r||_inf        (cycle start / restart)
//   cycle-start kernel  decides whether the cycle runs, g = beta e1
//   store (mode 1)      v_1 = r / beta, compressed into V[:,0]
//   per step j (all enqueued asynchronously, self-disabling once the cycle stops):
//     spmv     w = A M^{-1} v_j  (decode fused), omega = ||w||       (Arnoldi SpMV)
//     dot      h = V_j^T w                                           (CGS)
//     axpy     w1 = w - V_j h                                        (CGS)
//     dot      u = V_j^T w1                                          (re-orth.)
//     axpy     w2 = w1 - V_j u, ||w2||_2, ||w2||_inf                 (re-orth.)
//     store    h_{j+1,j} = ||w2||, Givens update, v_{j+1} -> V        (extension)
//   backsolve y = R^{-1} g; x += M^{-1} (V y)                        (LS update)
// The host reads the explicit residual once per cycle and polls a mapped flag every
// `check_every` steps to stop enqueueing once the device has ended the cycle.
//
// NVTX ranges (header-only NVTX 3; inert unless a profiler is attached) mark every
// restart cycle ("cbgmres cycle") and every launch by kernel class ("cbgmres basis_dot",
// "... basis_axpy", "... spmv", "... store", "... other"), so a profiler can select the
// launches of one class or one cycle.
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <new>
#include <utility>
#include <vector>

#include "../../include/cbgmres.h"
#include "cbg_launch.h"

using namespace cbg;

namespace {

#define CBG_CUDA(call)                                   \
    do {                                                 \
        cudaError_t e_ = (call);                         \
        if (e_ != cudaSuccess) {                         \
            last_cuda_error = e_;                        \
            return CBG_ERR_CUDA;                         \
        }                                                \
    } while (0)

thread_local cudaError_t last_cuda_error = cudaSuccess;

int fmt_bytes(int fmt)
{
    switch (fmt) {
    case CBG_F64: return 8;
    case CBG_F32: case CBG_I32: return 4;
    case CBG_F16: case CBG_BF16: case CBG_I16: return 2;
    case CBG_E4M3: return 1;
    default: return 0;
    }
}

int num_sms()
{
    static int sms = 0;
    if (!sms) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (sms <= 0) sms = 1;
    }
    return sms;
}

// ------------------------------------------------------------------ format dispatch
struct Ops {
    void (*dot)(int, int, cudaStream_t, const DotArgs&);
    void (*axpy)(int, int, int, cudaStream_t, const AxpyArgs&);
    void (*dot_tma)(int, cudaStream_t, const DotArgs&, int*);
    bool (*tma_fits)();
    void (*store)(int, cudaStream_t, const StoreArgs&);
    void (*spmv_code)(int, int, int, cudaStream_t, const SpmvArgs&);
    void (*spmv_sell)(int, cudaStream_t, const SellArgs&);
    void (*encode)(int, cudaStream_t, const double*, long long, unsigned char*, EncParams);
    void (*decode)(int, cudaStream_t, const unsigned char*, long long, double, double*);
    int (*occ_dot)();
    int (*occ_axpy)();
    int (*occ_spmv)();
};

template <int F> Ops make_ops()
{
    return Ops{&Launcher<F>::dot, &Launcher<F>::axpy, &Launcher<F>::dot_tma,
               &Launcher<F>::tma_fits, &Launcher<F>::store, &Launcher<F>::spmv_code, &Launcher<F>::spmv_sell,
               &Launcher<F>::encode, &Launcher<F>::decode, &Launcher<F>::occupancy_dot,
               &Launcher<F>::occupancy_axpy, &Launcher<F>::occupancy_spmv};
}

const Ops& ops_for(int fmt)
{
    static const Ops table[7] = {make_ops<F64>(), make_ops<F32>(), make_ops<F16>(), make_ops<BF16>(),
                                 make_ops<E4M3>(), make_ops<I32>(), make_ops<I16>()};
    return table[fmt];
}

long long round_up(long long a, long long b) { return (a + b - 1) / b * b; }

constexpr long long SPMV_TUNE_MIN_ROWS = 65536;   // create times the SpMV schedules from here on

// Next basis format of the adaptive ladder (options.adapt): e4m3 -> bf16 -> f32 -> f64,
// f16 -> f32, i16 -> i32 -> f64; -1 at the top.
int promote_format(int fmt)
{
    switch (fmt) {
    case CBG_E4M3: return CBG_BF16;
    case CBG_BF16: return CBG_F32;
    case CBG_F16: return CBG_F32;
    case CBG_I16: return CBG_I32;
    case CBG_F32: return CBG_F64;
    case CBG_I32: return CBG_F64;
    default: return -1;
    }
}

// --------------------------------------------------------------- small helper kernels
// a vector as double-float hi and lo planes (w for the dot kernels, the matrix values for
// the double-float SpMV)
__global__ void k_split_df(const double* w, long long n, float* out)
{
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        float h, l;
        split_f64(w[i], h, l);
        out[i] = h;
        out[n + i] = l;
    }
}

// largest |v| and smallest nonzero |v| as FP64 bit patterns (non-negative doubles order as
// integers); mm = {max, min} must start as {0, ~0}
__global__ void k_abs_range(const double* v, long long n, unsigned long long* mm)
{
    unsigned long long mx = 0ull, mn = ~0ull;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const unsigned long long b = (unsigned long long)__double_as_longlong(v[i]) & 0x7FFFFFFFFFFFFFFFull;
        mx = b > mx ? b : mx;
        if (b != 0ull) mn = b < mn ? b : mn;
    }
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long ox = __shfl_xor_sync(0xFFFFFFFFu, mx, o), on = __shfl_xor_sync(0xFFFFFFFFu, mn, o);
        mx = ox > mx ? ox : mx;
        mn = on < mn ? on : mn;
    }
    if ((threadIdx.x & 31) == 0) {
        if (mx) atomicMax(mm, mx);
        if (mn != ~0ull) atomicMin(mm + 1, mn);
    }
}

// out = the values times 2^e (exact) as double-float hi / lo planes
__global__ void k_split_df_pow2(const double* v, long long n, int e, float* out)
{
    const double sc = pow2d(e);
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        float h, l;
        split_f64(__dmul_rn(v[i], sc), h, l);
        out[i] = h;
        out[n + i] = l;
    }
}

// Sliced-ELL copy: entries per row of every chunk of 32 rows (a warp per chunk)
__global__ void k_sell_len(const int* rowptr, long long n, long long nchunks, int* len)
{
    const int lane = threadIdx.x & 31;
    for (long long c = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5; c < nchunks;
         c += ((long long)gridDim.x * blockDim.x) >> 5) {
        const long long row = c * 32 + lane;
        int l = row < n ? rowptr[row + 1] - rowptr[row] : 0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) l = max(l, __shfl_xor_sync(0xffffffffu, l, o));
        if (lane == 0) len[c] = l;
    }
}

// ... and the entries: the split values (CSR-order planes valdf[2 * nnz]) and columns in
// chunk order, padding with zero values and the row's own index (rows past n: column 0)
__global__ void k_sell_fill(const int* rowptr, const int* col, const float* valdf, long long nnz, long long n,
                            long long nchunks, const int* len, const long long* off, long long entries, int* scol,
                            float* sval)
{
    for (long long row = (long long)blockIdx.x * blockDim.x + threadIdx.x; row < nchunks * 32;
         row += (long long)gridDim.x * blockDim.x) {
        const long long c = row >> 5;
        const int lane = (int)(row & 31), L = len[c];
        const int p0 = row < n ? rowptr[row] : 0, cnt = row < n ? rowptr[row + 1] - p0 : 0;
        for (int k = 0; k < L; k++) {
            const long long q = off[c] + 32ll * k + lane;
            if (k < cnt) {
                scol[q] = col[p0 + k];
                sval[q] = valdf[p0 + k];
                sval[entries + q] = valdf[nnz + p0 + k];
            } else {
                scol[q] = row < n ? (int)row : 0;
                sval[q] = 0.f;
                sval[entries + q] = 0.f;
            }
        }
    }
}

__global__ void k_jacobi_prepare(const int* rowptr, const int* col, const double* val, long long n,
                                 double* dinv, int* bad)
{
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        double d = 0.0;
        for (int p = rowptr[i]; p < rowptr[i + 1]; p++)
            if (col[p] == i) d = val[p];
        if (d == 0.0 || !isfinite(d)) { atomicExch(bad, 1); dinv[i] = 0.0; }
        else dinv[i] = 1.0 / d;
    }
}

// Block-Jacobi with blocks of BJ rows (Section 5.5 uses block size 4): one thread per
// diagonal block extracts it from A, inverts it by Gauss-Jordan elimination with partial
// pivoting in FP64, and writes its rows of P = D^{-1} as a CSR matrix (rows of a full
// block hold BJ entries, the last block's rows hold its size).  A zero pivot (singular
// block) or a non-finite inverse sets *bad.
constexpr int BJ = 4;
__global__ void k_bj_setup(const int* rowptr, const int* col, const double* val, long long n, int* prow,
                           int* pcol, double* pval, int* bad)
{
    const long long nb = (n + BJ - 1) / BJ, nfull = n / BJ;
    for (long long b = (long long)blockIdx.x * blockDim.x + threadIdx.x; b < nb; b += (long long)gridDim.x * blockDim.x) {
        const long long r0 = b * BJ;
        const int kb = (int)(n - r0 < BJ ? n - r0 : BJ);
        double M[BJ][2 * BJ];
        for (int i = 0; i < kb; i++) {
            for (int k = 0; k < 2 * BJ; k++) M[i][k] = (k == kb + i) ? 1.0 : 0.0;
            for (int p = rowptr[r0 + i]; p < rowptr[r0 + i + 1]; p++) {
                const long long c = col[p] - r0;
                if (c >= 0 && c < kb) M[i][c] = val[p];
            }
        }
        bool ok = true;
        for (int k = 0; k < kb && ok; k++) {
            int piv = k;
            for (int i = k + 1; i < kb; i++)
                if (fabs(M[i][k]) > fabs(M[piv][k])) piv = i;
            if (M[piv][k] == 0.0) { ok = false; break; }
            if (piv != k)
                for (int c = 0; c < 2 * kb; c++) { const double t = M[k][c]; M[k][c] = M[piv][c]; M[piv][c] = t; }
            const double inv = 1.0 / M[k][k];
            for (int c = 0; c < 2 * kb; c++) M[k][c] = __dmul_rn(M[k][c], inv);
            for (int i = 0; i < kb; i++) {
                if (i == k) continue;
                const double f = M[i][k];
                if (f != 0.0)
                    for (int c = 0; c < 2 * kb; c++) M[i][c] = __fma_rn(-f, M[k][c], M[i][c]);
            }
        }
        for (int i = 0; i < kb; i++) {
            const long long row = r0 + i;
            const long long q = row < nfull * BJ ? row * BJ : nfull * BJ * BJ + (long long)(row - nfull * BJ) * kb;
            prow[row] = (int)q;
            for (int c = 0; c < kb; c++) {
                const double v = ok ? M[i][kb + c] : 0.0;
                if (!isfinite(v)) ok = false;
                pcol[q + c] = (int)(r0 + c);
                pval[q + c] = v;
            }
        }
        if (!ok) atomicExch(bad, 1);
        if (b == nb - 1) prow[n] = (int)(nfull * BJ * BJ + (long long)(n - nfull * BJ) * (n - nfull * BJ));
    }
}

__global__ void k_scale_columns(const int* col, const double* val, const double* dinv, long long nnz, double* out)
{
    for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < nnz; p += (long long)gridDim.x * blockDim.x)
        out[p] = __dmul_rn(val[p], dinv[col[p]]);
}

__global__ void k_init_state(DevState* st, double bnorm, double target, double eps_bd, int m, int record,
                             long long hist_cap)
{
    st->active = 0;
    st->k = 0;
    st->stop = 0;
    st->kcap = 0;
    st->m = m;
    st->record = record;
    st->iters = 0;
    st->reorths = 0;
    st->bnorm = bnorm;
    st->target = target;
    st->beta = 0.0;
    st->rinf = 0.0;
    st->omega = 0.0;
    st->eps_bd = eps_bd;
    st->est = 0.0;
    st->hn = 0.0;
    st->hist_cap = hist_cap;
    st->last_k = 0;
    st->fault = 0;
    st->reorth_now = 0;
}

// ================================================ cycle start / end (single block)
// start: decide whether a new cycle runs, reset g, counters of the cycle.
__global__ void k_cycle_start(DevArrays d, long long maxit, int m)
{
    if (threadIdx.x != 0) return;
    DevState* st = d.st;
    const double beta = st->beta;
    int run = beta > st->target && st->iters < maxit && isfinite(beta);
    long long left = maxit - st->iters;
    st->kcap = (int)(left < m ? left : m);
    st->last_k = st->k;
    st->k = 0;
    st->stop = 0;
    st->active = run;
    if (d.flag_host) *(volatile int*)d.flag_host = run;
    for (int i = 0; i <= m; i++) { d.g[i] = 0.0; d.y[i] = 0.0; }
    d.g[0] = beta;
}

// y = R^{-1} g on the k x k upper triangle (the least-squares step of Fig. 1); one warp, column-oriented:
// y_c = g_c / R_cc, then g_i -= R_ic y_c for i < c (lanes split i; column c is
// contiguous).  The next column is prefetched while the current one is applied.
__global__ void k_backsolve(DevArrays d)
{
    __shared__ double gs[MAXCOLS + 1];
    DevState* st = d.st;
    const int k = st->k, ldh = st->m + 1;
    const int lane = threadIdx.x;
    for (int i = lane; i <= st->m; i += 32) gs[i] = i < k ? d.g[i] : 0.0;
    __syncwarp();
    constexpr int PER = (MAXCOLS + 31) / 32;
    double cur[PER], nxt[PER];
    if (k > 0) {
        const double* col = d.R + (long long)(k - 1) * ldh;
#pragma unroll
        for (int t = 0; t < PER; t++) { int i = lane + 32 * t; cur[t] = i < k ? col[i] : 0.0; }
    }
    for (int c = k - 1; c >= 0; c--) {
        if (c > 0) {
            const double* col = d.R + (long long)(c - 1) * ldh;
#pragma unroll
            for (int t = 0; t < PER; t++) { int i = lane + 32 * t; nxt[t] = i < c ? col[i] : 0.0; }
        }
        // R_cc sits in lane c % 32, slot c / 32
        double rcc = 0.0;
#pragma unroll
        for (int t = 0; t < PER; t++) if (t == c / 32) rcc = cur[t];
        rcc = __shfl_sync(0xFFFFFFFFu, rcc, c % 32);
        const double yc = gs[c] / rcc;
        __syncwarp();
#pragma unroll
        for (int t = 0; t < PER; t++) {
            int i = lane + 32 * t;
            if (i < c) gs[i] = __dsub_rn(gs[i], __dmul_rn(cur[t], yc));
        }
        if (lane == 0) gs[c] = yc;
        __syncwarp();
#pragma unroll
        for (int t = 0; t < PER; t++) cur[t] = nxt[t];
    }
    for (int i = lane; i <= st->m; i += 32) d.y[i] = i < k ? gs[i] : 0.0;
}

// ||v||_2 and finiteness of a vector: per-block partials, last block combines them in a
// fixed order.  out[0] = norm, out[1] = 1 if all entries are finite.
__global__ void __launch_bounds__(THREADS) k_vec_norm(const double* v, long long n, double* part,
                                                      unsigned int* counter, double* out)
{
    __shared__ double red[THREADS / 32];
    __shared__ int fin;
    if (threadIdx.x == 0) fin = 1;
    __syncthreads();
    double s = 0.0;
    int ok = 1;
    for (long long i = (long long)blockIdx.x * THREADS + threadIdx.x; i < n; i += (long long)gridDim.x * THREADS) {
        double x = v[i];
        if (!isfinite(x)) ok = 0;
        s = __fma_rn(x, x, s);
    }
    if (!ok) fin = 0;
    s = warp_sum(s);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < THREADS / 32; w++) t += red[w];
        part[2 * blockIdx.x] = t;
        part[2 * blockIdx.x + 1] = fin;
    }
    if (last_block(counter)) {
        if (threadIdx.x < 32) {
            double t = 0.0, f = 1.0;
            for (unsigned int b = threadIdx.x; b < gridDim.x; b += 32) {
                t += __ldcg(part + 2 * b);
                f = fmin(f, __ldcg(part + 2 * b + 1));
            }
            t = warp_sum(t);
            for (int o = 16; o > 0; o >>= 1) f = fmin(f, __shfl_xor_sync(0xFFFFFFFFu, f, o));
            if (threadIdx.x == 0) {
                out[0] = sqrt(t);
                out[1] = f;
            }
        }
    }
}

}  // namespace

// last CUDA error seen by the library on this thread (cbgmres_last_error)
void cbg_record_cuda_error(cudaError_t e) { last_cuda_error = e; }

// ======================================================================== the handle
struct cbg_handle {
    long long n = 0, nnz = 0, ld = 0, ldb = 0;
    int m = 0, fmt = 0;
    cbg_options opt{};
    cudaStream_t stream = nullptr;
    // matrix
    int* rowptr = nullptr;
    int* col = nullptr;
    double* val = nullptr;     // A
    double* valp = nullptr;    // A D^{-1} (Jacobi) or nullptr
    float* valdf = nullptr;    // the Arnoldi SpMV's values (valp or val) times 2^pexp as FP32
                               // hi / lo planes, or null (FP64 products)
    int pexp = 0;              // the per-step operator is normalised by 2^pexp
    double* dinv = nullptr;    // D^{-1}
    double* pvals = nullptr;   // values of P: SPAI (A's pattern) or block-Jacobi inverse blocks
    int* prow = nullptr;       // P's pattern: A's for SPAI, the diagonal blocks for block-Jacobi
    int* pcol = nullptr;
    bool own_ppat = false;
    // basis and vectors
    unsigned char* V = nullptr;
    double *w = nullptr, *w1 = nullptr, *w2 = nullptr, *r = nullptr, *tmp = nullptr, *z = nullptr;
    double* wdf = nullptr;    // w (then w1) split into FP32 hi[ld] and lo[ld] planes for the DF32 dot
    double *bdev = nullptr, *xdev = nullptr;   // staging for cbgmres_solve_host
    double* scratch = nullptr;                 // small reductions
    // solver state
    DevArrays d{};
    void* state_block = nullptr;
    int* flag_host = nullptr;
    int* flag_dev = nullptr;
    long long hist_alloc = 0;
    int grid_dot = 0, grid_axpy = 0, grid_store = 0, grid_spmv = 0, group = 1, gridmax = 0;
    int grid_tma = 0;         // bulk-copy pipelined basis kernels: one block per SM
    int fmt0 = 0;             // the handle's basis format (options.adapt may move up from it)
    bool use_tma = false;
    // sliced-ELL copy of the per-step operator (chunks of 32 rows), used when the
    // create-time timing finds it faster than the CSR SpMV
    int* sell_len = nullptr;
    long long* sell_off = nullptr;
    int* sell_col = nullptr;
    float* sell_val = nullptr;
    long long sell_entries = 0, sell_chunks = 0;
    bool use_sell = false;
    int grid_sell = 0;
    int test_stall = 0;            // cbgmres_test_stall: pipelined dots still to be stalled
    long long test_wait = 0;       //   and their wait limit in clock cycles
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    std::vector<cudaEvent_t> step_ev;
    // launch accounting and optional per-kernel profiling
    long long launches = 0;
    std::vector<cudaEvent_t> prof_ev;      // pool of event pairs
    std::vector<int> prof_cls;             // class of each recorded pair
    std::vector<double> prof_bytes;        // algorithmic bytes of each pair
    int prof_used = 0;
    cbg_profile prof{};
};

namespace {

void dfree(void* p);

void free_handle(cbg_handle* h)
{
    if (!h) return;
    dfree(h->rowptr); dfree(h->col); dfree(h->val); dfree(h->valp); dfree(h->valdf); dfree(h->dinv);
    if (h->own_ppat) { dfree(h->prow); dfree(h->pcol); }
    dfree(h->pvals); dfree(h->V); dfree(h->w); dfree(h->wdf); dfree(h->w1); dfree(h->w2); dfree(h->r);
    dfree(h->tmp); dfree(h->z); dfree(h->bdev); dfree(h->xdev); dfree(h->scratch);
    dfree(h->sell_len); dfree(h->sell_off); dfree(h->sell_col); dfree(h->sell_val);
    dfree(h->state_block);
    if (h->d.hist) {   // stream-ordered allocation (see run_solve); the frees above synchronised
        cudaFreeAsync(h->d.hist, 0);
        cudaStreamSynchronize(0);
    }
    if (h->flag_host) cudaFreeHost(h->flag_host);
    if (h->ev0) cudaEventDestroy(h->ev0);
    if (h->ev1) cudaEventDestroy(h->ev1);
    for (auto e : h->step_ev) cudaEventDestroy(e);
    for (auto e : h->prof_ev) cudaEventDestroy(e);
    delete h;
}

int validate_csr_host(long long n, long long nnz, const int* rp, const int* ci)
{
    if (rp[0] != 0 || rp[n] != nnz) return CBG_ERR_ARG;
    for (long long i = 0; i < n; i++)
        if (rp[i + 1] < rp[i]) return CBG_ERR_ARG;
    for (long long p = 0; p < nnz; p++)
        if (ci[p] < 0 || ci[p] >= n) return CBG_ERR_ARG;
    return CBG_OK;
}

#ifdef CBG_DEBUG
// Debug build (-DCBG_DEBUG): every device allocation of this file carries a guard tail of
// GUARD_BYTES bytes of 0xA5 after the bytes asked for; cbgmres_solve checks every live
// guard after each solve, and cbgmres_debug_guard_check on demand.
constexpr size_t GUARD_BYTES = 4096;
constexpr unsigned char GUARD_FILL = 0xA5;
std::mutex g_guard_mu;
std::vector<std::pair<void*, size_t>> g_guards;   // (base, bytes before the guard)
thread_local const char* debug_message = nullptr;
#endif

template <class T> int dalloc(T** p, size_t count)
{
    if (count == 0) count = 1;
    const size_t bytes = count * sizeof(T);
#ifdef CBG_DEBUG
    cudaError_t e = cudaMalloc((void**)p, bytes + GUARD_BYTES);
    if (e == cudaSuccess) e = cudaMemset(reinterpret_cast<unsigned char*>(*p) + bytes, GUARD_FILL, GUARD_BYTES);
    if (e == cudaSuccess) {
        std::lock_guard<std::mutex> lk(g_guard_mu);
        g_guards.emplace_back(static_cast<void*>(*p), bytes);
    }
#else
    cudaError_t e = cudaMalloc((void**)p, bytes);
#endif
    if (e != cudaSuccess) {
        *p = nullptr;
        last_cuda_error = e;
        return e == cudaErrorMemoryAllocation ? CBG_ERR_OOM : CBG_ERR_CUDA;
    }
    return CBG_OK;
}

// cudaFree for memory from dalloc (the debug build also forgets its guard)
void dfree(void* p)
{
#ifdef CBG_DEBUG
    if (p) {
        std::lock_guard<std::mutex> lk(g_guard_mu);
        for (size_t i = 0; i < g_guards.size(); i++)
            if (g_guards[i].first == p) {
                g_guards.erase(g_guards.begin() + (long)i);
                break;
            }
    }
#endif
    cudaFree(p);
}

#ifdef CBG_DEBUG
// CBG_OK when every live guard still holds its fill pattern
int check_guards()
{
    std::vector<unsigned char> buf(GUARD_BYTES);
    std::lock_guard<std::mutex> lk(g_guard_mu);
    for (const auto& g : g_guards) {
        if (cudaMemcpy(buf.data(), static_cast<unsigned char*>(g.first) + g.second, GUARD_BYTES,
                       cudaMemcpyDeviceToHost) != cudaSuccess)
            return CBG_ERR_CUDA;
        for (unsigned char c : buf)
            if (c != GUARD_FILL) {
                debug_message = "debug build: a device write ran past the end of a library allocation";
                return CBG_ERR_CUDA;
            }
    }
    return CBG_OK;
}
#endif

int spmv_grid(long long n, int group, int sms, int occ)
{
    return std::max(1, (int)std::min<long long>((n * group + THREADS - 1) / THREADS, (long long)sms * occ));
}

int pick_group(long long n, long long nnz)
{
    double mean = n > 0 ? (double)nnz / (double)n : 1.0;
    if (mean < 10) return 1;
    if (mean < 20) return 4;
    if (mean < 48) return 8;
    if (mean < 96) return 16;
    return 32;
}

// ------------------------------------------------------------- profiling of launches
// Every library launch goes through `launch`, which counts it and, with profiling on,
// brackets it with a pair of events recorded on the handle's stream.
void harvest_profile(cbg_handle* h)
{
    // all recorded pairs precede a completed stream synchronisation
    for (int i = 0; i < h->prof_used; i++) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, h->prof_ev[2 * i], h->prof_ev[2 * i + 1]) == cudaSuccess) {
            const int c = h->prof_cls[i];
            h->prof.ms[c] += ms;
            h->prof.bytes[c] += h->prof_bytes[i];
            h->prof.launches[c] += 1;
        }
    }
    h->prof_used = 0;
}

const char* const kClassRange[5] = {"cbgmres basis_dot", "cbgmres basis_axpy", "cbgmres spmv", "cbgmres store",
                                     "cbgmres other"};

template <class F> void launch(cbg_handle* h, int cls, double bytes, F&& f)
{
    h->launches++;
    const bool prof = h->opt.profile && h->prof_used < (int)h->prof_cls.size();
    if (prof) cudaEventRecord(h->prof_ev[2 * h->prof_used], h->stream);
    nvtxRangePushA(kClassRange[cls]);
    f();
    nvtxRangePop();
    if (prof) {
        cudaEventRecord(h->prof_ev[2 * h->prof_used + 1], h->stream);
        h->prof_cls[h->prof_used] = cls;
        h->prof_bytes[h->prof_used] = bytes;
        h->prof_used++;
    }
}

// algorithmic HBM bytes of one SpMV (CSR values + indices + row pointers, x read, y
// written) and of one store (w read, codes written)
double spmv_bytes(const cbg_handle* h)
{
    return (double)h->nnz * 12.0 + (double)(h->n + 1) * 4.0 + 16.0 * (double)h->n;
}
double store_bytes(const cbg_handle* h) { return (double)h->n * (8.0 + (double)fmt_bytes(h->fmt)); }

// ------------------------------------------------------------------ launches per step
// Basis format of the following cycles: code stride and the format-dependent grids.
void set_format(cbg_handle* h, int fmt)
{
    const Ops& op = ops_for(fmt);
    const int sms = num_sms();
    h->fmt = fmt;
    h->ldb = h->ld * fmt_bytes(fmt);
    h->grid_dot = std::max(1, (int)std::min<long long>(h->ld / DOT_MIN_ROWS, (long long)sms * std::max(1, op.occ_dot())));
    const long long axpy_blocks = h->ld / ((long long)THREADS * (16 / fmt_bytes(fmt)));
    h->grid_axpy = std::max(1, (int)std::min<long long>(axpy_blocks, (long long)sms * std::max(1, op.occ_axpy())));
}

SellArgs sell_args(cbg_handle* h, const void* x, const double* xscale_dev, float* ydf, const int* active)
{
    SellArgs a{};
    a.len = h->sell_len;
    a.off = h->sell_off;
    a.col = h->sell_col;
    a.val = h->sell_val;
    a.entries = h->sell_entries;
    a.nchunks = h->sell_chunks;
    a.n = h->n;
    a.x = x;
    a.xscale_dev = xscale_dev;
    a.ydf = ydf;
    a.ydf_ld = h->ld;
    a.part = h->d.part_spmv;
    a.counter = h->d.counters + 1;
    a.st = h->d.st;
    a.active = active;
    return a;
}

SpmvArgs spmv_args(cbg_handle* h)
{
    SpmvArgs a{};
    a.rowptr = h->rowptr;
    a.col = h->col;
    a.n = h->n;
    a.part = h->d.part_spmv;
    a.st = h->d.st;
    return a;
}

void enqueue_residual(cbg_handle* h, const double* b, const double* x)
{
    SpmvArgs a = spmv_args(h);
    a.val = h->val;
    a.x = x;
    a.xscale = 1.0;
    a.b = b;
    a.y = h->r;
    a.counter = h->d.counters + 0;
    launch(h, 2, spmv_bytes(h), [&] { spmv_f64(SPMV_RESIDUAL, h->group, h->grid_spmv, h->stream, a); });
}

// The modified Gram-Schmidt variant Section 2 names in place of CGS: within a pass,
// column i's coefficient comes from w as columns 0..i-1 have already reduced it, and
// w -= h_i v_i follows at once.  That is 2(j+1) dependent launches per pass (one-column
// dot, one-column axpy) where CGS takes 2, each re-reading and re-writing w: the paper's
// reason to prefer CGS.  DF32 keeps w as its double-float planes, reduced in place; FP64
// alternates w between two buffers.  The final axpy writes w2 and finalises its norms
// for the store kernel, like the CGS path.
template <class Dot, class Axpy>
void enqueue_mgs(cbg_handle* h, int j, bool reorth, float* wdf, DotArgs& da, AxpyArgs& xa, Dot&& run_dot,
                 Axpy&& run_axpy)
{
    const int passes = reorth ? 2 : 1;
    const double col_bytes = (double)h->n * (double)fmt_bytes(h->fmt);
    double* cur = h->w;                       // FP64 arithmetic: the current w
    for (int pass = 0; pass < passes; pass++) {
        double* coef = pass == 0 ? h->d.h : h->d.u;
        da.counter = h->d.counters + (pass == 0 ? 2 : 3);
        for (int i = 0; i <= j; i++) {
            const bool last = pass == passes - 1 && i == j;
            da.V = h->V + (long long)i * h->ldb;
            da.ncols = 1;
            da.scales = h->d.scales + i;
            da.w = cur;
            da.out = coef + i;
            launch(h, 0, col_bytes, run_dot);
            xa.V = da.V;
            xa.ncols = 1;
            xa.scales = da.scales;
            xa.coef = coef + i;
            double* next = last ? h->w2 : (cur == h->w1 ? h->w : h->w1);
            xa.w_in = wdf ? nullptr : cur;
            xa.wdf_in = wdf;
            xa.wdf_out = last ? nullptr : wdf;
            xa.w_out = next;
            xa.counter = last ? h->d.counters + 5 : nullptr;
            launch(h, 1, col_bytes, [&] { run_axpy(xa); });
            cur = next;
        }
    }
}

void enqueue_step(cbg_handle* h, int j)
{
    const Ops& op = ops_for(h->fmt);
    cudaStream_t s = h->stream;
    const int* active = &h->d.st->active;
    const unsigned char* Vj = h->V + (long long)j * h->ldb;
    float* wdf = h->opt.arith == CBG_ARITH_DF32 ? reinterpret_cast<float*>(h->wdf) : nullptr;
    // w = A M^{-1} v_j, omega
    {
        SpmvArgs a = spmv_args(h);
        a.active = active;
        a.xscale_dev = h->d.scales + j;
        a.x = Vj;
        if (h->opt.precond == CBG_PC_SPAI || h->opt.precond == CBG_PC_BJ4) {
            a.rowptr = h->prow;
            a.col = h->pcol;
            a.val = h->pvals;
            a.y = h->z;
            launch(h, 2, spmv_bytes(h), [&] { op.spmv_code(SPMV_PLAIN, h->group, h->grid_spmv, s, a); });   // z = P v
            SpmvArgs b2 = spmv_args(h);
            b2.active = active;
            b2.val = h->val;
            b2.x = h->z;
            b2.xscale = 1.0;
            b2.y = h->w;
            b2.ydf = wdf;
            b2.ydf_ld = h->ld;
            b2.valdf = wdf ? h->valdf : nullptr;
            b2.nnz = h->nnz;
            b2.counter = h->d.counters + 1;
            if (h->use_sell && wdf) {
                SellArgs sa2 = sell_args(h, h->z, nullptr, wdf, active);
                launch(h, 2, spmv_bytes(h), [&] { spmv_sell_f64(h->grid_sell, s, sa2); });                // w = A z
            } else {
                launch(h, 2, spmv_bytes(h), [&] { spmv_f64(SPMV_ARNOLDI, h->group, h->grid_spmv, s, b2); });   // w = A z
            }
        } else {
            a.val = h->valp ? h->valp : h->val;
            a.y = h->w;
            a.ydf = wdf;
            a.ydf_ld = h->ld;
            a.valdf = wdf ? h->valdf : nullptr;
            a.nnz = h->nnz;
            a.xexp = a.valdf ? 0 : h->pexp;          // (the planes hold the scaled values)
            a.counter = h->d.counters + 1;
            if (h->use_sell && wdf) {
                SellArgs sa1 = sell_args(h, Vj, h->d.scales + j, wdf, active);
                launch(h, 2, spmv_bytes(h), [&] { op.spmv_sell(h->grid_sell, s, sa1); });
            } else {
                launch(h, 2, spmv_bytes(h), [&] { op.spmv_code(SPMV_ARNOLDI, h->group, h->grid_spmv, s, a); });
            }
        }
    }
    const int ncols = j + 1;
    const bool reorth = h->opt.reorth != CBG_REORTH_NEVER;
    const bool cond = h->opt.reorth == CBG_REORTH_CONDITIONAL;   // Fig. 1: when ||w1|| < eta omega
    const double pass_bytes = (double)ncols * (double)h->n * (double)fmt_bytes(h->fmt);
    // CGS: h = V^T w ; w1 = w - V h
    DotArgs da{};
    da.V = h->V;
    da.ldb = h->ldb;
    da.ncols = ncols;
    da.scales = h->d.scales;
    da.nrows = h->ld;
    da.part = h->d.part;
    da.active = active;
    da.w = h->w;
    da.wdf = wdf;
    da.counter = h->d.counters + 2;
    da.out = h->d.h;
    // DF32: the bulk-copy pipelined dot (one block per SM); FP64 keeps the register kernel
    auto run_dot = [&] {
        if (h->use_tma) {
            DotArgs dt = da;
            if (h->test_stall > 0) {          // cbgmres_test_stall: this launch times out
                dt.withhold = 1;
                dt.wait_limit = h->test_wait;
                h->test_stall--;
            }
            op.dot_tma(h->grid_tma, s, dt, &h->d.st->fault);
        } else {
            op.dot(h->opt.arith, h->grid_dot, s, da);
        }
    };
    auto run_axpy = [&](const AxpyArgs& xa) { op.axpy(h->opt.arith, EPI_SUB, h->grid_axpy, s, xa); };
    AxpyArgs xa{};
    xa.V = h->V;
    xa.ldb = h->ldb;
    xa.ncols = ncols;
    xa.scales = h->d.scales;
    xa.sign = -1.0;
    xa.nrows = h->ld;
    xa.n = h->n;
    xa.part_norm = h->d.part_norm;
    xa.active = active;
    xa.st = h->d.st;                                      // the final pass writes ||w||, max |w| here
    if (h->opt.ortho == CBG_ORTHO_MGS) {
        enqueue_mgs(h, j, reorth, wdf, da, xa, run_dot, run_axpy);
    } else {
        launch(h, 0, pass_bytes, run_dot);
        xa.coef = h->d.h;
        // DF32: the SpMV delivered w only as its double-float planes
        xa.w_in = wdf ? nullptr : h->w;
        xa.wdf_in = wdf;
        xa.w_out = reorth ? h->w1 : h->w2;
        // the final pass finalises the norms; in conditional mode the first pass does too,
        // and its last block decides on the device whether the second pass runs
        xa.counter = reorth && !cond ? nullptr : h->d.counters + 5;
        xa.wdf_out = reorth ? wdf : nullptr;                  // the second dot reads w1 split
        // DF32, second pass always: w1 is read only as its split planes (by the second dot
        // and the second axpy), so the first axpy writes nothing else
        const bool planes_only = reorth && !cond && wdf;
        if (planes_only) xa.w_out = nullptr;
        if (cond) {
            xa.reorth_flag = &h->d.st->reorth_now;
            xa.eta = h->opt.eta;
        }
        launch(h, 1, pass_bytes, [&] { run_axpy(xa); });
        if (reorth) {
            // re-orthogonalisation: u = V^T w1 ; w2 = w1 - V u ; (h += u in the store kernel);
            // conditional mode: both kernels skip themselves unless the flag is set
            const int* gate = cond ? &h->d.st->reorth_now : active;
            da.w = h->w1;
            da.counter = h->d.counters + 3;
            da.out = h->d.u;
            da.active = gate;
            launch(h, 0, pass_bytes, run_dot);
            xa.coef = h->d.u;
            xa.w_in = planes_only ? nullptr : h->w1;
            xa.wdf_in = planes_only ? wdf : nullptr;
            xa.w_out = h->w2;
            xa.wdf_out = nullptr;
            xa.counter = h->d.counters + 5;
            xa.reorth_flag = nullptr;
            xa.active = gate;
            launch(h, 1, pass_bytes, [&] { run_axpy(xa); });
        }
    }
    // h_{j+1,j}, breakdown test, basis extension and the Givens update
    StoreArgs sa{};
    sa.d = h->d;
    sa.w = h->w2;
    sa.Vcol = h->V + (long long)(j + 1) * h->ldb;
    sa.col = j + 1;
    sa.j = j;
    sa.mode = 0;
    sa.reorth = reorth ? 1 : 0;
    sa.n = h->n;
    sa.fmt = h->fmt;
    sa.counter = h->d.counters + 6;
    sa.hexp = -h->pexp;
    if (cond) {
        sa.reorth_dev = &h->d.st->reorth_now;
        sa.w_alt = h->w1;
    }
    launch(h, 3, store_bytes(h), [&] { op.store(h->grid_store, s, sa); });
}

void enqueue_first_vector(cbg_handle* h)
{
    StoreArgs sa{};
    sa.d = h->d;
    sa.w = h->r;
    sa.Vcol = h->V;
    sa.col = 0;
    sa.j = 0;
    sa.mode = 1;
    sa.n = h->n;
    sa.fmt = h->fmt;
    launch(h, 3, store_bytes(h), [&] { ops_for(h->fmt).store(h->grid_store, h->stream, sa); });
}

void enqueue_cycle_end(cbg_handle* h, double* x)
{
    cudaStream_t s = h->stream;
    launch(h, 4, 0.0, [&] { k_backsolve<<<1, 32, 0, s>>>(h->d); });
    const Ops& op = ops_for(h->fmt);
    AxpyArgs xa{};
    xa.V = h->V;
    xa.ldb = h->ldb;
    xa.ncols = 0;
    xa.ncols_dev = &h->d.st->k;
    xa.scales = h->d.scales;
    xa.coef = h->d.y;
    xa.sign = 1.0;
    xa.nrows = h->ld;
    xa.n = h->n;
    auto run_axpy = [&](int epi) { op.axpy(h->opt.arith, epi, h->grid_axpy, s, xa); };
    if (h->opt.precond == CBG_PC_SPAI || h->opt.precond == CBG_PC_BJ4) {
        xa.w_out = h->tmp;
        launch(h, 4, 0.0, [&] { run_axpy(EPI_PLAIN); });                                          // t = V y
        SpmvArgs a = spmv_args(h);
        a.rowptr = h->prow;
        a.col = h->pcol;
        a.val = h->pvals;
        a.x = h->tmp;
        a.xscale = 1.0;
        a.y = x;
        launch(h, 4, 0.0, [&] { spmv_f64(SPMV_ACCUM, h->group, h->grid_spmv, s, a); });           // x += P t
    } else {
        xa.w_out = x;
        xa.dinv = h->opt.precond == CBG_PC_JACOBI ? h->dinv : nullptr;
        launch(h, 4, 0.0, [&] { run_axpy(EPI_XUPD); });                                           // x += D^{-1} V y
    }
}

struct HostState {
    DevState st;
};

int read_state(cbg_handle* h, DevState* out)
{
    CBG_CUDA(cudaMemcpyAsync(out, h->d.st, sizeof(DevState), cudaMemcpyDeviceToHost, h->stream));
    CBG_CUDA(cudaStreamSynchronize(h->stream));
    if (out->fault == FAULT_BOUNDS) {          // debug build: an index out of range was skipped
#ifdef CBG_DEBUG
        debug_message = "debug build: a CSR column index out of range was skipped by the SpMV";
#endif
        return CBG_ERR_ARG;
    }
    if (out->fault) return CBG_ERR_TIMEOUT;   // a pipelined kernel stopped waiting
    return CBG_OK;
}

// The whole solve; x (device) holds x0 on entry.  k_only > 0: stop after the first
// cycle with at most k_only steps (Arnoldi parity runs).
int run_solve(cbg_handle* h, const double* b, double* x, double tol, long long maxit, cbg_stats* stats,
              int k_only)
{
    if (!h || !b || !x || !(tol >= 0.0) || maxit < 0) return CBG_ERR_ARG;
    cudaStream_t s = h->stream;
    if (h->fmt != h->fmt0) set_format(h, h->fmt0);   // every solve starts in the handle's format
    long long promotions = 0;
    CBG_CUDA(cudaEventRecord(h->ev0, s));
    // ||b|| and finiteness of b and x0
    const long long launches0 = h->launches;
    launch(h, 4, 0.0, [&] {
        k_vec_norm<<<h->grid_spmv, THREADS, 0, s>>>(b, h->n, h->d.part_spmv, h->d.counters + 4, h->scratch);
    });
    launch(h, 4, 0.0, [&] {
        k_vec_norm<<<h->grid_spmv, THREADS, 0, s>>>(x, h->n, h->d.part_spmv, h->d.counters + 4, h->scratch + 2);
    });
    double nb[4];
    CBG_CUDA(cudaMemcpyAsync(nb, h->scratch, 4 * sizeof(double), cudaMemcpyDeviceToHost, s));
    CBG_CUDA(cudaStreamSynchronize(s));
    CBG_CUDA(cudaGetLastError());
    const double bnorm = nb[0];
    int status = CBG_OK;
    long long cycles = 0;
    double bytes = 0.0;
    DevState hs{};
    const long long hist_cap = stats && stats->history && stats->history_cap > 0 ? stats->history_cap : 0;
    if (nb[1] == 0.0 || nb[3] == 0.0) {
        status = CBG_ERR_NONFINITE;
    } else if (bnorm == 0.0) {
        CBG_CUDA(cudaMemsetAsync(x, 0, h->n * sizeof(double), s));
    } else {
        if (hist_cap > h->hist_alloc) {
            // stream-ordered, so growing the history buffer does not synchronise the device
            if (h->d.hist) CBG_CUDA(cudaFreeAsync(h->d.hist, s));
            h->d.hist = nullptr;
            h->hist_alloc = 0;
            cudaError_t e = cudaMallocAsync((void**)&h->d.hist, (size_t)hist_cap * sizeof(double), s);
            if (e != cudaSuccess) {
                h->d.hist = nullptr;
                last_cuda_error = e;
                return e == cudaErrorMemoryAllocation ? CBG_ERR_OOM : CBG_ERR_CUDA;
            }
            h->hist_alloc = hist_cap;
        }
        const double target = tol * bnorm;
        const long long maxit_eff = k_only > 0 ? std::min<long long>(maxit, k_only) : maxit;
        launch(h, 4, 0.0, [&] {
            k_init_state<<<1, 1, 0, s>>>(h->d.st, bnorm, target, h->opt.breakdown_eps, h->m, hist_cap > 0,
                                         hist_cap);
        });
        const double spmv_bytes = (double)h->nnz * 12.0 + (double)(h->n + 1) * 4.0 + 16.0 * (double)h->n;
        const int L = (int)h->step_ev.size();
        long long iters_before = -1;
        double prev_beta = INFINITY;
        bool stagnated = false;
        for (;;) {
            enqueue_residual(h, b, x);
            launch(h, 4, 0.0, [&] { k_cycle_start<<<1, 1, 0, s>>>(h->d, maxit_eff, h->m); });
            int rc = read_state(h, &hs);
            if (rc) return rc;
            harvest_profile(h);
            for (int j = 0; j < hs.last_k; j++)
                bytes += spmv_bytes + 4.0 * (double)(j + 1) * (double)h->n * (double)fmt_bytes(h->fmt);
            if (!hs.active) break;
            if (k_only > 0 && cycles >= 1) break;
            if (cycles > 0 && hs.iters == iters_before) return CBG_ERR_CUDA;   // no progress: device work failed
            if (h->opt.stop_on_stagnation && cycles > 0 && !(hs.beta < prev_beta)) {
                stagnated = true;
                break;
            }
            // adaptive basis format: the compressed basis lost more accuracy in the last
            // cycle than its recurrence residual accounts for -> next format of the ladder
            if (h->opt.adapt && cycles > 0 && hs.beta > h->opt.adapt_gap * hs.est) {
                const int nf = promote_format(h->fmt);
                if (nf >= 0) {
                    set_format(h, nf);
                    promotions++;
                }
            }
            prev_beta = hs.beta;
            iters_before = hs.iters;
            cycles++;
            nvtxRangePushA("cbgmres cycle");
            enqueue_first_vector(h);
            const int kcap = hs.kcap;
            for (int j = 0; j < kcap; j++) {
                if (j >= L) {
                    // keep at most L steps in flight; stop enqueueing once the cycle ended
                    if (cudaEventSynchronize(h->step_ev[j % L]) != cudaSuccess) {
                        nvtxRangePop();
                        CBG_CUDA(cudaGetLastError());
                        return CBG_ERR_CUDA;
                    }
                    if (*(volatile int*)h->flag_host == 0) break;
                }
                enqueue_step(h, j);
                if (cudaEventRecord(h->step_ev[j % L], s) != cudaSuccess) {
                    nvtxRangePop();
                    CBG_CUDA(cudaGetLastError());
                    return CBG_ERR_CUDA;
                }
            }
            enqueue_cycle_end(h, x);
            nvtxRangePop();
            CBG_CUDA(cudaGetLastError());
        }
        if (!std::isfinite(hs.beta)) status = CBG_ERR_NONFINITE;
        else if (hs.beta <= hs.target) status = CBG_OK;
        else status = stagnated ? CBG_STAGNATED : CBG_NOT_CONVERGED;
    }
    CBG_CUDA(cudaEventRecord(h->ev1, s));
    CBG_CUDA(cudaEventSynchronize(h->ev1));
    CBG_CUDA(cudaGetLastError());
    harvest_profile(h);
    if (stats) {
        stats->kernel_launches = h->launches - launches0;
        float ms = 0.f;
        cudaEventElapsedTime(&ms, h->ev0, h->ev1);
        stats->iters = hs.iters;
        stats->restarts = cycles;
        stats->reorths = hs.reorths;
        stats->true_relres = bnorm > 0 ? hs.beta / bnorm : 0.0;
        stats->est_relres = bnorm > 0 ? hs.est / bnorm : 0.0;
        stats->ms_total = ms;
        stats->bytes_model = bytes;
        stats->status = status;
        stats->fmt_final = h->fmt;
        stats->promotions = promotions;
        stats->history_len = 0;
        if (hist_cap > 0 && bnorm > 0) {
            long long nh = std::min<long long>(hs.iters, hist_cap);
            if (nh > 0)
                CBG_CUDA(cudaMemcpy(stats->history, h->d.hist, nh * sizeof(double), cudaMemcpyDeviceToHost));
            stats->history_len = nh;
        }
    }
    return status;
}

}  // namespace

// ======================================================================== C ABI
extern "C" {

void cbgmres_options_default(cbg_options* o)
{
    if (!o) return;
    std::memset(o, 0, sizeof(*o));
    o->reorth = CBG_REORTH_ALWAYS;
    o->precond = CBG_PC_NONE;
    o->arith = CBG_ARITH_DF32;
    o->spmv_group = 0;
    o->eta = 0.70710678118654752440;
    o->breakdown_eps = 1.4210854715202004e-14;   // 2^-46
    o->stream = nullptr;
    o->check_every = 4;
    o->use_graph = 0;
    o->profile = 0;
    o->stop_on_stagnation = 0;
    o->adapt = 0;
    o->adapt_gap = 4.0;
}

const char* cbgmres_status_string(int s)
{
    switch (s) {
    case CBG_OK: return "converged";
    case CBG_NOT_CONVERGED: return "not converged within maxit";
    case CBG_STAGNATED: return "stagnated (explicit residual did not decrease over a restart)";
    case CBG_ERR_ARG: return "invalid argument";
    case CBG_ERR_NONFINITE: return "non-finite value";
    case CBG_ERR_OOM: return "device out of memory";
    case CBG_ERR_CUDA: return "CUDA error";
    case CBG_ERR_TIMEOUT: return "device wait timed out";
    case CBG_ERR_UNSUPPORTED: return "unsupported combination";
    default: return "unknown status";
    }
}

int cbgmres_format_bytes(int fmt) { return fmt_bytes(fmt); }

const char* cbgmres_last_error(void)
{
#ifdef CBG_DEBUG
    if (debug_message) return debug_message;
#endif
    return last_cuda_error == cudaSuccess ? "no CUDA error" : cudaGetErrorString(last_cuda_error);
}

int cbgmres_create(const cbg_csr* A, int restart, int fmt, const cbg_options* opt, cbg_handle** out)
{
    if (!out) return CBG_ERR_ARG;
    *out = nullptr;
    if (!A || A->n < 1 || A->nnz < 1 || A->n > 0x7FFFFFFFLL || A->nnz > 0x7FFFFFFFLL || restart < 1 ||
        restart + 1 > MAXCOLS || fmt_bytes(fmt) == 0 || !A->row_ptr || !A->col || !A->val)
        return CBG_ERR_ARG;
    cbg_options o;
    if (opt) o = *opt;
    else cbgmres_options_default(&o);
    if (o.arith != CBG_ARITH_DF32 && o.arith != CBG_ARITH_FP64) return CBG_ERR_ARG;
    if (o.precond < CBG_PC_NONE || o.precond > CBG_PC_BJ4) return CBG_ERR_ARG;
    if (o.reorth < CBG_REORTH_ALWAYS || o.reorth > CBG_REORTH_NEVER) return CBG_ERR_ARG;
    if (o.ortho != CBG_ORTHO_CGS && o.ortho != CBG_ORTHO_MGS) return CBG_ERR_ARG;
    if (o.reorth == CBG_REORTH_CONDITIONAL && o.ortho == CBG_ORTHO_MGS) return CBG_ERR_UNSUPPORTED;
    if (o.reorth == CBG_REORTH_CONDITIONAL && !(o.eta > 0.0 && o.eta <= 1.0)) return CBG_ERR_ARG;
    if (o.spmv_group != 0 && o.spmv_group != -1 &&
        (o.spmv_group < 1 || o.spmv_group > 32 || (o.spmv_group & (o.spmv_group - 1))))
        return CBG_ERR_ARG;

    // validate the CSR on the host
    const long long n = A->n, nnz = A->nnz;
    std::vector<int> hrp, hci;
    const int* rp = A->row_ptr;
    const int* ci = A->col;
    if (A->on_device) {
        hrp.resize(n + 1);
        hci.resize(nnz);
        if (cudaMemcpy(hrp.data(), A->row_ptr, (n + 1) * sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess ||
            cudaMemcpy(hci.data(), A->col, nnz * sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess)
            return CBG_ERR_CUDA;
        rp = hrp.data();
        ci = hci.data();
    }
    if (validate_csr_host(n, nnz, rp, ci)) return CBG_ERR_ARG;

    cbg_handle* h = new (std::nothrow) cbg_handle();
    if (!h) return CBG_ERR_OOM;
    h->n = n;
    h->nnz = nnz;
    h->m = restart;
    h->fmt = fmt;
    h->opt = o;
    h->stream = (cudaStream_t)o.stream;
    h->ld = round_up(n, TILE_ROWS);
    h->ldb = h->ld * fmt_bytes(fmt);
    int rc = CBG_OK;
#define TRY(x)                     \
    do {                           \
        rc = (x);                  \
        if (rc) {                  \
            free_handle(h);        \
            return rc;             \
        }                          \
    } while (0)
    const cudaMemcpyKind kind = A->on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    TRY(dalloc(&h->rowptr, n + 1));
    TRY(dalloc(&h->col, nnz));
    TRY(dalloc(&h->val, nnz));
    if (cudaMemcpy(h->rowptr, A->row_ptr, (n + 1) * sizeof(int), kind) != cudaSuccess ||
        cudaMemcpy(h->col, A->col, nnz * sizeof(int), kind) != cudaSuccess ||
        cudaMemcpy(h->val, A->val, nnz * sizeof(double), kind) != cudaSuccess)
        TRY(CBG_ERR_CUDA);
    TRY(dalloc(&h->scratch, 64));
    if (o.precond == CBG_PC_JACOBI) {
        TRY(dalloc(&h->dinv, h->ld));
        TRY(dalloc(&h->valp, nnz));
        int* bad = (int*)h->scratch;
        cudaMemset(bad, 0, sizeof(int));
        k_jacobi_prepare<<<1024, 256>>>(h->rowptr, h->col, h->val, n, h->dinv, bad);
        k_scale_columns<<<2048, 256>>>(h->col, h->val, h->dinv, nnz, h->valp);
        int hbad = 0;
        if (cudaMemcpy(&hbad, bad, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) TRY(CBG_ERR_CUDA);
        if (hbad) TRY(CBG_ERR_ARG);
    }
    // The per-step operator (A D^{-1} under Jacobi, else A) is normalised by a power of two,
    // 2^pexp, so that its largest |value| lies in [1, 2): w = A v then stays near unit size
    // and the double-float products and sums of squares stay far from FP32 underflow and
    // overflow whatever the matrix's scale.  The Hessenberg columns are scaled back
    // exactly.  (SPAI and block Jacobi apply an approximate inverse first: A P is already
    // normalised.)  Its values are split into double-float planes unless their dynamic
    // range exceeds 2^64 (FP64 products then).
    {
        const bool norm = o.precond == CBG_PC_NONE || o.precond == CBG_PC_JACOBI;
        const double* vs = h->valp ? h->valp : h->val;
        unsigned long long* mm = (unsigned long long*)h->scratch;
        const unsigned long long init[2] = {0ull, ~0ull};
        unsigned long long hm[2] = {0ull, 0ull};
        if (cudaMemcpy(mm, init, sizeof(init), cudaMemcpyHostToDevice) != cudaSuccess) TRY(CBG_ERR_CUDA);
        k_abs_range<<<1024, 256>>>(vs, nnz, mm);
        if (cudaMemcpy(hm, mm, sizeof(hm), cudaMemcpyDeviceToHost) != cudaSuccess) TRY(CBG_ERR_CUDA);
        double vmax = 0.0, vmin = 0.0;
        std::memcpy(&vmax, &hm[0], sizeof(double));
        std::memcpy(&vmin, &hm[1], sizeof(double));
        h->pexp = norm && vmax > 0.0 ? std::max(-960, std::min(960, -std::ilogb(vmax))) : 0;
        const double smax = std::ldexp(vmax, h->pexp), smin = std::ldexp(vmin, h->pexp);
        if (vmax == 0.0 || (smin >= 0x1p-64 && smax <= 0x1p32)) {
            TRY(dalloc(&h->valdf, 2 * nnz));
            k_split_df_pow2<<<2048, 256>>>(vs, nnz, h->pexp, h->valdf);
        }
        if (cudaGetLastError() != cudaSuccess) TRY(CBG_ERR_CUDA);
    }
    h->prow = h->rowptr;
    h->pcol = h->col;
    if (o.precond == CBG_PC_BJ4) {
        const long long nfull = n / BJ, rest = n - nfull * BJ, pnnz = nfull * BJ * BJ + rest * rest;
        h->own_ppat = true;
        TRY(dalloc(&h->prow, n + 1));
        TRY(dalloc(&h->pcol, pnnz));
        TRY(dalloc(&h->pvals, pnnz));
        int* bad = (int*)h->scratch;
        cudaMemset(bad, 0, sizeof(int));
        k_bj_setup<<<(int)std::min<long long>((n / BJ + 256) / 256, 4096), 256>>>(h->rowptr, h->col, h->val, n,
                                                                                  h->prow, h->pcol, h->pvals, bad);
        int hbad = 0;
        if (cudaMemcpy(&hbad, bad, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) TRY(CBG_ERR_CUDA);
        if (hbad) TRY(CBG_ERR_ARG);
    }
    // the adaptive ladder may end at f64: room for 8-byte codes
    const size_t vbytes = (size_t)(restart + 1) * h->ld * (o.adapt ? 8 : fmt_bytes(fmt));
    TRY(dalloc(&h->V, vbytes));
    if (cudaMemset(h->V, 0, vbytes) != cudaSuccess) TRY(CBG_ERR_CUDA);
    double** vecs[] = {&h->w, &h->w1, &h->w2, &h->r, &h->tmp, &h->z, &h->wdf};
    for (double** p : vecs) {
        TRY(dalloc(p, h->ld));
        if (cudaMemset(*p, 0, h->ld * sizeof(double)) != cudaSuccess) TRY(CBG_ERR_CUDA);
    }

    // launch geometry (format-dependent parts: set_format; with options.adapt the
    // per-block partial arrays are sized for every format of the ladder)
    const int sms = num_sms();
    // one grid for every SpMV of the handle: the least occupancy of the FP64-vector kernels
    // and of the per-step kernels of every format the handle may use, so that no SpMV
    // launch spills into a partial second wave
    int occ_min = spmv_occupancy();
    for (int f = fmt; f >= 0; f = o.adapt ? promote_format(f) : -1) occ_min = std::min(occ_min, ops_for(f).occ_spmv());
    const int occ_spmv = std::max(1, occ_min);
    h->fmt0 = fmt;
    h->grid_store = (int)std::min<long long>((n + THREADS - 1) / THREADS, (long long)sms * 4);
    h->group = o.spmv_group > 0 ? o.spmv_group : pick_group(n, nnz);
    h->grid_spmv = spmv_grid(n, h->group, sms, occ_spmv);
    h->grid_store = std::max(1, h->grid_store);
    h->grid_tma = sms;
    h->use_tma = o.arith == CBG_ARITH_DF32;
    // (room for the SpMV partials of every lane count the create-time tuning may pick)
    h->gridmax = std::max(std::max(h->grid_store, spmv_grid(n, 32, sms, occ_spmv)), h->grid_tma);
    for (int f = fmt; f >= 0; f = o.adapt ? promote_format(f) : -1) {
        if (o.arith == CBG_ARITH_DF32 && !ops_for(f).tma_fits()) TRY(CBG_ERR_UNSUPPORTED);
        set_format(h, f);
        h->gridmax = std::max(h->gridmax, std::max(h->grid_dot, h->grid_axpy));
    }
    set_format(h, fmt);

    // state block: DevState + H, R, cs, sn, g, y, h, u, scales + partials + counters
    const int m = restart, ldh = m + 1;
    size_t off = 0;
    auto take = [&](size_t bytes) {
        size_t o2 = off;
        off += (bytes + 255) / 256 * 256;
        return o2;
    };
    size_t o_st = take(sizeof(DevState));
    size_t o_H = take(sizeof(double) * ldh * m), o_R = take(sizeof(double) * ldh * m);
    size_t o_cs = take(sizeof(double) * m), o_sn = take(sizeof(double) * m);
    size_t o_g = take(sizeof(double) * ldh), o_y = take(sizeof(double) * ldh);
    size_t o_h = take(sizeof(double) * ldh), o_u = take(sizeof(double) * ldh);
    size_t o_sc = take(sizeof(double) * ldh);
    size_t o_part = take(sizeof(double) * (size_t)h->gridmax * MAXCOLS);
    size_t o_pn = take(sizeof(double) * (size_t)h->gridmax * 2);
    size_t o_ps = take(sizeof(double) * (size_t)h->gridmax * 2);
    size_t o_cnt = take(sizeof(unsigned int) * 16);
    unsigned char* blk = nullptr;
    TRY(dalloc(&blk, off));
    h->state_block = blk;
    if (cudaMemset(blk, 0, off) != cudaSuccess) TRY(CBG_ERR_CUDA);
    h->d.st = (DevState*)(blk + o_st);
    h->d.H = (double*)(blk + o_H);
    h->d.R = (double*)(blk + o_R);
    h->d.cs = (double*)(blk + o_cs);
    h->d.sn = (double*)(blk + o_sn);
    h->d.g = (double*)(blk + o_g);
    h->d.y = (double*)(blk + o_y);
    h->d.h = (double*)(blk + o_h);
    h->d.u = (double*)(blk + o_u);
    h->d.scales = (double*)(blk + o_sc);
    h->d.part = (double*)(blk + o_part);
    h->d.part_norm = (double*)(blk + o_pn);
    h->d.part_spmv = (double*)(blk + o_ps);
    h->d.counters = (unsigned int*)(blk + o_cnt);
    h->d.hist = nullptr;
    if (cudaHostAlloc((void**)&h->flag_host, sizeof(int), cudaHostAllocMapped) != cudaSuccess) TRY(CBG_ERR_CUDA);
    *h->flag_host = 0;
    if (cudaHostGetDevicePointer((void**)&h->flag_dev, h->flag_host, 0) != cudaSuccess) TRY(CBG_ERR_CUDA);
    h->d.flag_host = h->flag_dev;
    if (cudaEventCreate(&h->ev0) != cudaSuccess || cudaEventCreate(&h->ev1) != cudaSuccess) TRY(CBG_ERR_CUDA);
    const int L = std::max(1, o.check_every);
    h->step_ev.resize(L, nullptr);
    for (auto& e : h->step_ev)
        if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) TRY(CBG_ERR_CUDA);
    // Automatic SpMV schedule on large matrices: time the per-step SpMV with 1, 2, ..., 32
    // lanes per row on this matrix (on the zero first basis column; the access pattern
    // does not depend on the values), and on a sliced-ELL copy of the double-float values
    // when the padding stays below a quarter of the nonzeros, and keep the fastest (the
    // copy only when it beats every CSR schedule by 10 %; otherwise it is freed again).
    const bool tune_spmv = !o.spmv_group && n >= SPMV_TUNE_MIN_ROWS;
    if ((tune_spmv || o.spmv_group == -1) && h->valdf && o.arith == CBG_ARITH_DF32) {
        const long long nch = (n + 31) / 32;
        TRY(dalloc(&h->sell_len, nch));
        k_sell_len<<<(int)std::min<long long>((nch * 32 + 255) / 256, 4096), 256>>>(h->rowptr, n, nch, h->sell_len);
        std::vector<int> lens(nch);
        std::vector<long long> offs(nch);
        if (cudaMemcpy(lens.data(), h->sell_len, nch * sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess)
            TRY(CBG_ERR_CUDA);
        long long total = 0;
        for (long long c = 0; c < nch; c++) { offs[c] = total; total += 32ll * lens[c]; }
        if (total <= nnz + nnz / 4 && total < (1ll << 31)) {
            h->sell_entries = total;
            h->sell_chunks = nch;
            TRY(dalloc(&h->sell_off, nch));
            TRY(dalloc(&h->sell_col, total));
            TRY(dalloc(&h->sell_val, 2 * total));
            if (cudaMemcpy(h->sell_off, offs.data(), nch * sizeof(long long), cudaMemcpyHostToDevice) != cudaSuccess)
                TRY(CBG_ERR_CUDA);
            k_sell_fill<<<(int)std::min<long long>((nch * 32 + 255) / 256, 4096), 256>>>(
                h->rowptr, h->col, h->valdf, nnz, n, nch, h->sell_len, h->sell_off, total, h->sell_col, h->sell_val);
            if (cudaGetLastError() != cudaSuccess) TRY(CBG_ERR_CUDA);
            h->grid_sell = (int)std::max<long long>(1, std::min<long long>((nch + THREADS / 32 - 1) / (THREADS / 32),
                                                                          (long long)sms * occ_spmv));
        }
    }
    if (o.spmv_group == -1) {                      // the sliced-ELL copy, as asked
        if (h->sell_entries == 0) TRY(CBG_ERR_UNSUPPORTED);
        h->use_sell = true;
    }
    if (tune_spmv) {
        double one = 1.0;
        if (cudaMemcpy(h->d.scales, &one, sizeof(double), cudaMemcpyHostToDevice) != cudaSuccess) TRY(CBG_ERR_CUDA);
        cudaEvent_t t0 = nullptr, t1 = nullptr;
        if (cudaEventCreate(&t0) != cudaSuccess || cudaEventCreate(&t1) != cudaSuccess) TRY(CBG_ERR_CUDA);
        // the shortest of 5 single launches after one warm-up launch (a single launch
        // is 10-100 us here: the minimum is far less noisy than a mean); before each, a
        // write of up to 256 MiB of the (still zero) basis evicts the matrix from L2, as
        // the basis products do between two SpMVs of a solve
        const size_t flush = std::min<size_t>(vbytes, size_t(256) << 20);
        auto time_min = [&](auto&& launch, float& best_ms) -> bool {
            launch();
            best_ms = 1e30f;
            for (int rep = 0; rep < 5; rep++) {
                if (cudaMemsetAsync(h->V, 0, flush, h->stream) != cudaSuccess) return false;
                cudaEventRecord(t0, h->stream);
                launch();
                cudaEventRecord(t1, h->stream);
                float ms = 0.f;
                if (cudaEventSynchronize(t1) != cudaSuccess || cudaEventElapsedTime(&ms, t0, t1) != cudaSuccess)
                    return false;
                best_ms = std::min(best_ms, ms);
            }
            return true;
        };
        float best = 1e30f;
        int best_g = h->group;
        bool ok = true;
        const Ops& op = ops_for(fmt);
        for (int g = 1; g <= 32 && ok; g *= 2) {
            SpmvArgs a = spmv_args(h);
            a.xscale_dev = h->d.scales;
            a.x = h->V;
            a.val = h->valp ? h->valp : h->val;
            a.y = h->w;
            a.ydf = h->opt.arith == CBG_ARITH_DF32 ? reinterpret_cast<float*>(h->wdf) : nullptr;
            a.ydf_ld = h->ld;
            a.valdf = a.ydf ? h->valdf : nullptr;
            a.nnz = h->nnz;
            a.xexp = a.valdf ? 0 : h->pexp;
            a.counter = h->d.counters + 1;
            const int grid = spmv_grid(n, g, sms, occ_spmv);
            float ms = 0.f;
            ok = time_min([&] { op.spmv_code(SPMV_ARNOLDI, g, grid, h->stream, a); }, ms);
            if (ok && ms < best) { best = ms; best_g = g; }
        }
        if (ok && h->sell_entries > 0 && h->opt.arith == CBG_ARITH_DF32) {
            SellArgs sa = sell_args(h, h->V, h->d.scales, reinterpret_cast<float*>(h->wdf), nullptr);
            float ms = 0.f;
            ok = time_min([&] { op.spmv_sell(h->grid_sell, h->stream, sa); }, ms);
            // The copy costs 12 bytes per entry of device memory, and timed cold it looks
            // better than it runs inside a solve, where part of the matrix stays in L2
            // between two SpMVs (upwind stencil, 96^3 and 128^3: 8 % faster cold, 4 % slower
            // in the solve): keep it only when it beats the best CSR schedule by 10 %.
            if (ok && ms < 0.90f * best) h->use_sell = true;
        }
        cudaEventDestroy(t0);
        cudaEventDestroy(t1);
        if (!ok) TRY(CBG_ERR_CUDA);
        h->group = best_g;
        h->grid_spmv = spmv_grid(n, best_g, sms, occ_spmv);
        if (!h->use_sell) {                               // not chosen: give the copy back
            dfree(h->sell_len); dfree(h->sell_off); dfree(h->sell_col); dfree(h->sell_val);
            h->sell_len = nullptr; h->sell_off = nullptr; h->sell_col = nullptr; h->sell_val = nullptr;
            h->sell_entries = 0;
            h->sell_chunks = 0;
        }
    }
    if (o.profile) {
        const int pairs = 8 * restart + 64;
        h->prof_ev.resize(2 * pairs, nullptr);
        h->prof_cls.resize(pairs, 0);
        h->prof_bytes.resize(pairs, 0.0);
        for (auto& e : h->prof_ev)
            if (cudaEventCreate(&e) != cudaSuccess) TRY(CBG_ERR_CUDA);
    }
    if (cudaDeviceSynchronize() != cudaSuccess) TRY(CBG_ERR_CUDA);
#undef TRY
    *out = h;
    return CBG_OK;
}

int cbgmres_set_spai(cbg_handle* h, const double* pvals, int on_device)
{
    if (!h || !pvals || h->opt.precond == CBG_PC_BJ4) return CBG_ERR_ARG;
    if (!h->pvals) {
        int rc = dalloc(&h->pvals, h->nnz);
        if (rc) return rc;
    }
    CBG_CUDA(cudaMemcpyAsync(h->pvals, pvals, h->nnz * sizeof(double),
                             on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, h->stream));
    CBG_CUDA(cudaStreamSynchronize(h->stream));
    return CBG_OK;
}

int cbgmres_solve(cbg_handle* h, const double* b, double* x, double tol, int64_t maxit, cbg_stats* stats)
{
    if (!h) return CBG_ERR_ARG;
    if (h->opt.precond == CBG_PC_SPAI && !h->pvals) return CBG_ERR_ARG;
    const int rc = run_solve(h, b, x, tol, maxit, stats, 0);
#ifdef CBG_DEBUG
    if (rc >= 0) {
        const int g = check_guards();
        if (g) return g;
    }
#endif
    return rc;
}

int cbgmres_debug_guard_check(cbg_handle* h, int poke)
{
#ifdef CBG_DEBUG
    if (!h) return CBG_ERR_ARG;
    if (poke) {                      // overwrite the first guard byte of the basis (a test)
        std::lock_guard<std::mutex> lk(g_guard_mu);
        for (const auto& g : g_guards)
            if (g.first == static_cast<void*>(h->V))
                CBG_CUDA(cudaMemset(static_cast<unsigned char*>(g.first) + g.second, 0, 1));
    }
    return check_guards();
#else
    (void)h;
    (void)poke;
    return CBG_ERR_UNSUPPORTED;
#endif
}

int cbgmres_solve_host(cbg_handle* h, const double* b_host, double* x_host, double tol, int64_t maxit,
                       cbg_stats* stats)
{
    if (!h || !b_host || !x_host) return CBG_ERR_ARG;
    if (!h->bdev || !h->xdev) {
        int rc = h->bdev ? CBG_OK : dalloc(&h->bdev, h->ld);
        if (!rc && !h->xdev) rc = dalloc(&h->xdev, h->ld);
        if (rc) return rc;
    }
    CBG_CUDA(cudaMemcpyAsync(h->bdev, b_host, h->n * sizeof(double), cudaMemcpyHostToDevice, h->stream));
    CBG_CUDA(cudaMemcpyAsync(h->xdev, x_host, h->n * sizeof(double), cudaMemcpyHostToDevice, h->stream));
    int st = cbgmres_solve(h, h->bdev, h->xdev, tol, maxit, stats);
    if (st < 0) return st;
    CBG_CUDA(cudaMemcpyAsync(x_host, h->xdev, h->n * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    CBG_CUDA(cudaStreamSynchronize(h->stream));
    return st;
}

int cbgmres_arnoldi(cbg_handle* h, const double* b, const double* x0, int k, double* H_host, int* k_done)
{
    if (!h || !b || !x0 || k < 1 || k > h->m || !H_host || !k_done) return CBG_ERR_ARG;
    if (!h->xdev) {
        int rc0 = dalloc(&h->xdev, h->ld);
        if (rc0) return rc0;
        rc0 = dalloc(&h->bdev, h->ld);
        if (rc0) return rc0;
    }
    double* x = h->xdev;   // work copy: the caller's x0 stays untouched
    CBG_CUDA(cudaMemcpyAsync(x, x0, h->n * sizeof(double), cudaMemcpyDeviceToDevice, h->stream));
    int st = run_solve(h, b, x, 0.0, k, nullptr, k);
    if (st < 0) return st;
    DevState hs{};
    int rc = read_state(h, &hs);
    if (rc) return rc;
    // after the solve the residual kernel ran again; H of the first cycle is intact
    const int kd = std::min(k, std::max(0, (int)std::min<long long>(hs.iters, k)));
    std::vector<double> H((size_t)(h->m + 1) * h->m);
    CBG_CUDA(cudaMemcpy(H.data(), h->d.H, H.size() * sizeof(double), cudaMemcpyDeviceToHost));
    for (int c = 0; c < kd; c++)
        for (int i = 0; i <= kd; i++) H_host[i + (size_t)c * (kd + 1)] = H[i + (size_t)c * (h->m + 1)];
    *k_done = kd;
    return CBG_OK;
}

int cbgmres_basis_column(cbg_handle* h, int col, double* out)
{
    if (!h || col < 0 || col > h->m || !out) return CBG_ERR_ARG;
    double sc = 1.0;
    CBG_CUDA(cudaMemcpyAsync(&sc, h->d.scales + col, sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    CBG_CUDA(cudaStreamSynchronize(h->stream));
    ops_for(h->fmt).decode(std::max(1, (int)std::min<long long>((h->n + THREADS - 1) / THREADS, 4096)), h->stream,
                           h->V + (long long)col * h->ldb, h->n, sc, out);
    CBG_CUDA(cudaGetLastError());
    CBG_CUDA(cudaStreamSynchronize(h->stream));
    return CBG_OK;
}

int cbgmres_spmv_group(const cbg_handle* h) { return h ? (h->use_sell ? 0 : h->group) : CBG_ERR_ARG; }

int cbgmres_test_stall(cbg_handle* h, int dots, long long wait_cycles)
{
    if (!h || dots < 0 || wait_cycles < 1) return CBG_ERR_ARG;
    if (!h->use_tma) return CBG_ERR_UNSUPPORTED;
    h->test_stall = dots;
    h->test_wait = wait_cycles;
    return CBG_OK;
}

int cbgmres_profile(cbg_handle* h, cbg_profile* out, int reset)
{
    if (!h || !out) return CBG_ERR_ARG;
    *out = h->prof;
    if (reset) h->prof = cbg_profile{};
    return CBG_OK;
}

int cbgmres_spmv(cbg_handle* h, const double* x, double* y)
{
    if (!h || !x || !y) return CBG_ERR_ARG;
    SpmvArgs a = spmv_args(h);
    a.val = h->val;
    a.x = x;
    a.xscale = 1.0;
    a.y = y;
    spmv_f64(SPMV_PLAIN, h->group, h->grid_spmv, h->stream, a);
    CBG_CUDA(cudaGetLastError());
    CBG_CUDA(cudaStreamSynchronize(h->stream));
    return CBG_OK;
}

int cbgmres_solve_fallback(cbg_handle* const* hs, int nh, const double* b, double* x, double tol, int64_t maxit,
                           cbg_stats* stats, int* used)
{
    if (!hs || nh < 1 || !b || !x || maxit < 0) return CBG_ERR_ARG;
    long long n = -1;
    for (int i = 0; i < nh; i++) {
        if (!hs[i]) continue;
        if (n >= 0 && hs[i]->n != n) return CBG_ERR_ARG;
        n = hs[i]->n;
    }
    if (n < 0) return CBG_ERR_ARG;
    cbg_handle* h0 = nullptr;
    for (int i = 0; i < nh && !h0; i++) h0 = hs[i];
    double* x0 = nullptr;
    int rc = dalloc(&x0, n);
    if (rc) return rc;
    cbg_stats tot{};
    int status = CBG_NOT_CONVERGED, last = -1;
    long long left = maxit;
    for (int i = 0; i < nh && left >= 0; i++) {
        if (!hs[i]) continue;
        last = i;
        if (cudaMemcpyAsync(x0, x, n * sizeof(double), cudaMemcpyDeviceToDevice, h0->stream) != cudaSuccess) {
            dfree(x0);
            return CBG_ERR_CUDA;
        }
        cudaStreamSynchronize(h0->stream);
        cbg_stats st{};
        status = run_solve(hs[i], b, x, tol, left, &st, 0);
        tot.iters += st.iters;
        tot.restarts += st.restarts;
        tot.reorths += st.reorths;
        tot.ms_total += st.ms_total;
        tot.bytes_model += st.bytes_model;
        tot.kernel_launches += st.kernel_launches;
        tot.true_relres = st.true_relres;
        tot.est_relres = st.est_relres;
        left -= st.iters;
        if (status == CBG_OK) break;
        if (status == CBG_ERR_NONFINITE)   // restore the iterate this attempt started from
            cudaMemcpy(x, x0, n * sizeof(double), cudaMemcpyDeviceToDevice);
        else if (status < 0) break;
    }
    dfree(x0);
    if (used) *used = last;
    if (stats) {
        const double* hist = stats->history;
        long long cap = stats->history_cap;
        *stats = tot;
        stats->history = const_cast<double*>(hist);
        stats->history_cap = cap;
        stats->history_len = 0;
        stats->status = status;
    }
    return status;
}

void cbgmres_destroy(cbg_handle* h)
{
    if (h) cudaStreamSynchronize(h->stream);
    free_handle(h);
}

// ---------------------------------------------------------------- codec test kernels
int cbg_encode(int fmt, int64_t n, const double* v, double vmax, void* codes, double* scale_out, void* stream)
{
    if (fmt_bytes(fmt) == 0 || n < 0 || (n > 0 && (!v || !codes)) || !scale_out) return CBG_ERR_ARG;
    EncParams ep = enc_params(fmt, vmax);
    *scale_out = ep.scale;
    if (n == 0) return CBG_OK;
    cudaStream_t s = (cudaStream_t)stream;
    int grid = (int)std::min<long long>((n + THREADS - 1) / THREADS, 8192);
    ops_for(fmt).encode(grid, s, v, n, (unsigned char*)codes, ep);
    CBG_CUDA(cudaGetLastError());
    CBG_CUDA(cudaStreamSynchronize(s));
    return CBG_OK;
}

int cbg_decode(int fmt, int64_t n, const void* codes, double scale, double* out, void* stream)
{
    if (fmt_bytes(fmt) == 0 || n < 0 || (n > 0 && (!codes || !out))) return CBG_ERR_ARG;
    if (n == 0) return CBG_OK;
    cudaStream_t s = (cudaStream_t)stream;
    int grid = (int)std::min<long long>((n + THREADS - 1) / THREADS, 8192);
    ops_for(fmt).decode(grid, s, (const unsigned char*)codes, n, scale, out);
    CBG_CUDA(cudaGetLastError());
    CBG_CUDA(cudaStreamSynchronize(s));
    return CBG_OK;
}

// Standalone basis products (test access).  V must have ld % TILE_ROWS == 0 rows per
// column and zero padding; w / the output vector must have ld elements.
int cbg_basis_dot(int fmt, int arith, int64_t n, int ncols, const void* V, int64_t ld, const double* scales,
                  const double* w, double* hout, void* stream)
{
    if (fmt_bytes(fmt) == 0 || (arith != 0 && arith != 1) || n < 1 || ncols < 1 || ncols > MAXCOLS || !V ||
        ld < n || ld % TILE_ROWS || !scales || !w || !hout)
        return CBG_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    const Ops& op = ops_for(fmt);
    const bool tma = arith == CBG_ARITH_DF32;
    int grid = tma ? num_sms()
                   : (int)std::min<long long>(ld / DOT_MIN_ROWS, (long long)num_sms() * std::max(1, op.occ_dot()));
    double *part = nullptr, *sc = nullptr, *out = nullptr, *wdf = nullptr;
    unsigned int* cnt = nullptr;   // [0] last-block counter, [1] fault flag
    int rc = dalloc(&part, (size_t)grid * MAXCOLS);
    if (!rc) rc = dalloc(&sc, ncols);
    if (!rc) rc = dalloc(&out, ncols);
    if (!rc) rc = dalloc(&cnt, 2);
    if (!rc && tma) rc = dalloc(&wdf, ld);
    if (!rc) {
        cudaMemsetAsync(cnt, 0, 2 * sizeof(unsigned int), s);
        cudaMemcpyAsync(sc, scales, ncols * sizeof(double), cudaMemcpyHostToDevice, s);
        DotArgs a{};
        a.V = (const unsigned char*)V;
        a.ldb = ld * fmt_bytes(fmt);
        a.ncols = ncols;
        a.scales = sc;
        a.w = w;
        a.nrows = ld;
        a.part = part;
        a.counter = cnt;
        a.out = out;
        if (tma) {
            k_split_df<<<(int)std::min<long long>((ld + THREADS - 1) / THREADS, 4096), THREADS, 0, s>>>(
                w, ld, reinterpret_cast<float*>(wdf));
            a.wdf = reinterpret_cast<const float*>(wdf);
            op.dot_tma(grid, s, a, reinterpret_cast<int*>(cnt + 1));
        } else {
            op.dot(arith, grid, s, a);
        }
        unsigned int flags[2] = {0u, 0u};
        if (cudaGetLastError() != cudaSuccess ||
            cudaMemcpyAsync(hout, out, ncols * sizeof(double), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
            cudaMemcpyAsync(flags, cnt, sizeof(flags), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess)
            rc = CBG_ERR_CUDA;
        else if (flags[1])
            rc = CBG_ERR_TIMEOUT;
    }
    dfree(part); dfree(sc); dfree(out); dfree(cnt); dfree(wdf);
    return rc;
}

int cbg_basis_axpy(int fmt, int arith, int64_t n, int ncols, const void* V, int64_t ld, const double* scales,
                   const double* hcoef, double* w, void* stream)
{
    if (fmt_bytes(fmt) == 0 || (arith != 0 && arith != 1) || n < 1 || ncols < 1 || ncols > MAXCOLS || !V ||
        ld < n || ld % TILE_ROWS || !scales || !hcoef || !w)
        return CBG_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    const Ops& op = ops_for(fmt);
    const long long blocks = ld / ((long long)THREADS * (16 / fmt_bytes(fmt)));
    int grid = (int)std::min<long long>(blocks, (long long)num_sms() * std::max(1, op.occ_axpy()));
    double *sc = nullptr, *cf = nullptr, *pn = nullptr;
    int rc = dalloc(&sc, ncols);
    if (!rc) rc = dalloc(&cf, ncols);
    if (!rc) rc = dalloc(&pn, (size_t)grid * 2);
    if (!rc) {
        cudaMemcpyAsync(sc, scales, ncols * sizeof(double), cudaMemcpyHostToDevice, s);
        cudaMemcpyAsync(cf, hcoef, ncols * sizeof(double), cudaMemcpyHostToDevice, s);
        AxpyArgs a{};
        a.V = (const unsigned char*)V;
        a.ldb = ld * fmt_bytes(fmt);
        a.ncols = ncols;
        a.scales = sc;
        a.coef = cf;
        a.sign = -1.0;
        a.w_in = w;
        a.w_out = w;
        a.nrows = ld;
        a.n = n;
        a.part_norm = pn;
        op.axpy(arith, EPI_SUB, grid, s, a);
        if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(s) != cudaSuccess) rc = CBG_ERR_CUDA;
    }
    dfree(sc); dfree(cf); dfree(pn);
    return rc;
}



}  // extern "C"
