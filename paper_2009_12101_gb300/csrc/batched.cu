// batched.cu -- host side of the batched persistent solve (C ABI in cbgmres.h).
//
// create: validate and pack every system (row pointers, local column indices, values,
// A D^{-1} and D^{-1} for Jacobi), order the work queue by decreasing size, allocate
// every basis once.  solve: replay a CUDA graph [set b/x pointers, clear the queue head,
// launch k_batched] and copy the per-system results back.  tune: time every candidate
// schedule (cluster size x split threshold) on the caller's problem and keep the fastest;
// results are cached in a small JSON-lines file keyed by GPU, format, restart length,
// system count and total rows.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <fstream>
#include <new>
#include <numeric>
#include <sstream>
#include <string>
#include <vector>

#include "../../include/cbgmres.h"
#include "cbg_launch.h"

using namespace cbg;

void cbg_record_cuda_error(cudaError_t e);   // solver.cu

namespace {

struct Schedule {
    int cluster = 1;
    int split_rows = 1 << 30;
    int lanes = 1;           // SpMV lanes per row (1: a thread per row)
};

template <int F> struct BOps {
    static cudaError_t launch(int c, int g, size_t sm, cudaStream_t s, const BatchArgs& a)
    {
        return Launcher<F>::batched(c, g, sm, s, a);
    }
    static int clusters(int c, size_t sm) { return Launcher<F>::batched_max_clusters(c, sm); }
};

cudaError_t launch_batched(int fmt, int c, int g, size_t sm, cudaStream_t s, const BatchArgs& a)
{
    switch (fmt) {
    case CBG_F64: return BOps<F64>::launch(c, g, sm, s, a);
    case CBG_F32: return BOps<F32>::launch(c, g, sm, s, a);
    case CBG_F16: return BOps<F16>::launch(c, g, sm, s, a);
    case CBG_BF16: return BOps<BF16>::launch(c, g, sm, s, a);
    case CBG_E4M3: return BOps<E4M3>::launch(c, g, sm, s, a);
    case CBG_I32: return BOps<I32>::launch(c, g, sm, s, a);
    default: return BOps<I16>::launch(c, g, sm, s, a);
    }
}

int max_clusters(int fmt, int c, size_t sm)
{
    switch (fmt) {
    case CBG_F64: return BOps<F64>::clusters(c, sm);
    case CBG_F32: return BOps<F32>::clusters(c, sm);
    case CBG_F16: return BOps<F16>::clusters(c, sm);
    case CBG_BF16: return BOps<BF16>::clusters(c, sm);
    case CBG_E4M3: return BOps<E4M3>::clusters(c, sm);
    case CBG_I32: return BOps<I32>::clusters(c, sm);
    default: return BOps<I16>::clusters(c, sm);
    }
}

int fbytes(int fmt) { return cbgmres_format_bytes(fmt); }

}  // namespace

struct cbg_batch {
    int nsys = 0, m = 0, fmt = 0;
    cbg_options opt{};
    cudaStream_t stream = nullptr;
    long long total_rows = 0, total_nnz = 0;
    int max_n = 0;
    std::vector<BatchSys> sys;
    std::vector<int> order;
    BatchSys* d_sys = nullptr;
    int* d_order = nullptr;
    int *d_rowptr = nullptr, *d_col = nullptr;
    double *d_val = nullptr, *d_valp = nullptr, *d_dinv = nullptr;
    float* d_valpdf = nullptr;   // the per-step SpMV's values as FP32 hi / lo planes (or null)
    unsigned char* d_V = nullptr;
    BatchOut* d_out = nullptr;
    unsigned int* d_queue = nullptr;
    double** d_io = nullptr;     // device table {b, x}
    double** h_io = nullptr;     // pinned host copy
    Schedule sched;
    bool have_graph = false;
    cudaGraphExec_t graph = nullptr;
    Schedule graph_sched;
    double graph_tol = -1.0;
    long long graph_maxit = -1;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaStream_t capture = nullptr;   // private stream for graph capture (the caller's may be
                                      // the legacy default stream, which cannot be captured)
    long long launches = 0;
};

namespace {

size_t smem_bytes(const cbg_batch* bt, const Schedule& sc)
{
    // rows of w one block holds: a cluster share of the largest cooperative system, or a
    // whole small system
    long long rows_cluster = sc.cluster > 1 ? ((bt->max_n + sc.cluster - 1) / sc.cluster + 15) / 16 * 16 : 0;
    long long rows_small = 0;
    for (const auto& s : bt->sys)
        if (sc.cluster == 1 || s.n < sc.split_rows) rows_small = std::max<long long>(rows_small, s.n);
    long long rows = std::max(rows_cluster, rows_small);
    return sizeof(BtSmem) + (size_t)(rows + 32) * sizeof(float2);
}

// Per system: the power of two 2^s that brings the largest |value| of its per-step operator
// into [1, 2), and whether that normalised operator's smallest nonzero |value| is at least
// 2^-64 (its double-float products then stay far from FP32 underflow).
int normalising_exponent(const double* v, long long n, bool& df_ok)
{
    double vmax = 0.0, vmin = INFINITY;
    for (long long p = 0; p < n; p++) {
        const double a = std::fabs(v[p]);
        vmax = std::max(vmax, a);
        if (a != 0.0) vmin = std::min(vmin, a);
    }
    if (vmax == 0.0) return 0;
    const int e = std::max(-960, std::min(960, -std::ilogb(vmax)));
    if (std::ldexp(vmin, e) < 0x1p-64) df_ok = false;
    return e;
}

// The values times 2^e (exact) as FP32 planes hi[n] then lo[n] with hi = RN(x) and
// lo = RN(x - hi) (the difference is exact in FP64), so |hi + lo - x| <= 2^-48 |x|.
void split_values_df(const double* v, long long n, int e, float* hi, float* lo)
{
    for (long long p = 0; p < n; p++) {
        const double x = std::ldexp(v[p], e);
        const float h = (float)x;
        hi[p] = h;
        lo[p] = (float)(x - (double)h);
    }
}

void free_batch(cbg_batch* bt)
{
    if (!bt) return;
    cudaFree(bt->d_sys); cudaFree(bt->d_order); cudaFree(bt->d_rowptr); cudaFree(bt->d_col);
    cudaFree(bt->d_val); cudaFree(bt->d_valp); cudaFree(bt->d_dinv); cudaFree(bt->d_valpdf);
    cudaFree(bt->d_V); cudaFree(bt->d_out);
    cudaFree(bt->d_queue); cudaFree(bt->d_io);
    if (bt->h_io) cudaFreeHost(bt->h_io);
    if (bt->graph) cudaGraphExecDestroy(bt->graph);
    if (bt->e0) cudaEventDestroy(bt->e0);
    if (bt->e1) cudaEventDestroy(bt->e1);
    if (bt->capture) cudaStreamDestroy(bt->capture);
    delete bt;
}

BatchArgs make_args(const cbg_batch* bt, const Schedule& sc, double tol, long long maxit)
{
    BatchArgs a{};
    a.sys = bt->d_sys;
    a.order = bt->d_order;
    a.nsys = bt->nsys;
    a.m = bt->m;
    a.rowptr = bt->d_rowptr;
    a.col = bt->d_col;
    a.valp = bt->d_valp ? bt->d_valp : bt->d_val;
    a.val = bt->d_val;
    a.dinv = bt->d_dinv;
    a.valpdf = bt->d_valpdf;
    a.nnz_all = bt->total_nnz;
    a.io = bt->d_io;
    a.V = bt->d_V;
    a.out = bt->d_out;
    a.queue = bt->d_queue;
    a.tol = tol;
    a.maxit = maxit;
    a.eps_bd = bt->opt.breakdown_eps;
    a.split_rows = sc.split_rows;
    a.max_rows_block = 0;
    a.spmv_lanes = sc.lanes;
    return a;
}

int grid_for(const cbg_batch* bt, const Schedule& sc, size_t sm)
{
    int nc = max_clusters(bt->fmt, sc.cluster, sm);
    if (nc <= 0) return 0;
    return nc * sc.cluster;
}

// enqueue one batched solve: pointer table, queue head, persistent kernel (grid and
// shared memory precomputed by grid_for, which also sets the kernel attributes, so that
// nothing but stream work happens here -- it may run under stream capture)
int enqueue(cbg_batch* bt, const Schedule& sc, int grid, size_t sm, double tol, long long maxit, cudaStream_t st)
{
    if (grid <= 0) return CBG_ERR_UNSUPPORTED;
    cudaError_t e = cudaMemcpyAsync(bt->d_io, bt->h_io, 2 * sizeof(double*), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(bt->d_queue, 0, sizeof(unsigned int), st);
    if (e == cudaSuccess) e = launch_batched(bt->fmt, sc.cluster, grid, sm, st, make_args(bt, sc, tol, maxit));
    if (e != cudaSuccess) {
        cbg_record_cuda_error(e);
        return CBG_ERR_CUDA;
    }
    bt->launches++;
    return CBG_OK;
}

int run_graph(cbg_batch* bt, double tol, long long maxit)
{
    const bool stale = !bt->have_graph || bt->graph_sched.cluster != bt->sched.cluster ||
                       bt->graph_sched.split_rows != bt->sched.split_rows ||
                       bt->graph_sched.lanes != bt->sched.lanes || bt->graph_tol != tol ||
                       bt->graph_maxit != maxit;
    if (stale) {
        if (bt->graph) cudaGraphExecDestroy(bt->graph);
        bt->graph = nullptr;
        bt->have_graph = false;
        cudaGraph_t g = nullptr;
        const size_t sm = smem_bytes(bt, bt->sched);
        const int grid = grid_for(bt, bt->sched, sm);
        if (grid <= 0) return CBG_ERR_UNSUPPORTED;
        cudaError_t ec = cudaStreamBeginCapture(bt->capture, cudaStreamCaptureModeRelaxed);
        if (ec != cudaSuccess) { cbg_record_cuda_error(ec); return CBG_ERR_CUDA; }
        int rc = enqueue(bt, bt->sched, grid, sm, tol, maxit, bt->capture);
        ec = cudaStreamEndCapture(bt->capture, &g);
        if (rc) {
            if (g) cudaGraphDestroy(g);
            return rc;
        }
        if (ec != cudaSuccess) { cbg_record_cuda_error(ec); return CBG_ERR_CUDA; }
        ec = cudaGraphInstantiate(&bt->graph, g, 0);
        cudaGraphDestroy(g);
        if (ec != cudaSuccess) { cbg_record_cuda_error(ec); return CBG_ERR_CUDA; }
        bt->have_graph = true;
        bt->graph_sched = bt->sched;
        bt->graph_tol = tol;
        bt->graph_maxit = maxit;
    }
    cudaError_t el = cudaGraphLaunch(bt->graph, bt->stream);
    if (el != cudaSuccess) { cbg_record_cuda_error(el); return CBG_ERR_CUDA; }
    return CBG_OK;
}

std::string tune_key(const cbg_batch* bt)
{
    cudaDeviceProp p{};
    int dev = 0;
    cudaGetDevice(&dev);
    cudaGetDeviceProperties(&p, dev);
    std::ostringstream os;
    os << p.name << "|sm" << p.major << p.minor << "|fmt" << bt->fmt << "|m" << bt->m << "|nsys" << bt->nsys
       << "|rows" << bt->total_rows << "|maxn" << bt->max_n;
    return os.str();
}

bool cache_lookup(const char* path, const std::string& key, Schedule* out)
{
    if (!path) return false;
    std::ifstream f(path);
    std::string line;
    bool found = false;
    while (std::getline(f, line)) {
        // {"key": "...", "cluster": C, "split_rows": S, "lanes": L}
        auto kp = line.find("\"key\": \"");
        if (kp == std::string::npos) continue;
        auto ke = line.find('"', kp + 8);
        if (line.substr(kp + 8, ke - kp - 8) != key) continue;
        int c = 0, s = 0;
        auto cp = line.find("\"cluster\": ");
        auto sp = line.find("\"split_rows\": ");
        if (cp == std::string::npos || sp == std::string::npos) continue;
        c = std::atoi(line.c_str() + cp + 11);
        s = std::atoi(line.c_str() + sp + 14);
        auto lp = line.find("\"lanes\": ");
        const int l = lp == std::string::npos ? 1 : std::atoi(line.c_str() + lp + 9);
        if (c >= 1 && s >= 1 && (l == 1 || l == 2 || l == 4 || l == 8)) {
            out->cluster = c;
            out->split_rows = s;
            out->lanes = l;
            found = true;   // the last entry for a key wins
        }
    }
    return found;
}

void cache_store(const char* path, const std::string& key, const Schedule& sc, double ms)
{
    if (!path) return;
    std::ofstream f(path, std::ios::app);
    f << "{\"key\": \"" << key << "\", \"cluster\": " << sc.cluster << ", \"split_rows\": " << sc.split_rows
      << ", \"lanes\": " << sc.lanes << ", \"ms\": " << ms << "}\n";
}

}  // namespace

extern "C" {

int cbgmres_create_batched(int nsys, const cbg_csr* As, int restart, int fmt, const cbg_options* opt,
                           cbg_batch** out)
{
    if (!out) return CBG_ERR_ARG;
    *out = nullptr;
    if (nsys < 1 || !As || restart < 1 || restart > BT_MAXM || fbytes(fmt) == 0) return CBG_ERR_ARG;
    cbg_options o;
    if (opt) o = *opt;
    else cbgmres_options_default(&o);
    if (o.precond != CBG_PC_NONE && o.precond != CBG_PC_JACOBI) return CBG_ERR_UNSUPPORTED;
    if (o.reorth != CBG_REORTH_ALWAYS || o.arith != CBG_ARITH_DF32 || o.ortho != CBG_ORTHO_CGS)
        return CBG_ERR_UNSUPPORTED;
    cbg_batch* bt = new (std::nothrow) cbg_batch();
    if (!bt) return CBG_ERR_OOM;
    bt->nsys = nsys;
    bt->m = restart;
    bt->fmt = fmt;
    bt->opt = o;
    bt->stream = (cudaStream_t)o.stream;
    // pack on the host (device CSRs are copied down first)
    std::vector<int> rp_all, ci_all;
    std::vector<double> va_all, vp_all, di_all;
    long long v_off = 0, vec_off = 0;
    const long long bs = fbytes(fmt);
    for (int s = 0; s < nsys; s++) {
        const cbg_csr& A = As[s];
        if (A.n < 1 || A.nnz < 1 || A.n > (1 << 28) || !A.row_ptr || !A.col || !A.val) { free_batch(bt); return CBG_ERR_ARG; }
        std::vector<int> rp(A.n + 1), ci(A.nnz);
        std::vector<double> va(A.nnz);
        const cudaMemcpyKind k = A.on_device ? cudaMemcpyDeviceToHost : cudaMemcpyHostToHost;
        if (cudaMemcpy(rp.data(), A.row_ptr, (A.n + 1) * sizeof(int), k) != cudaSuccess ||
            cudaMemcpy(ci.data(), A.col, A.nnz * sizeof(int), k) != cudaSuccess ||
            cudaMemcpy(va.data(), A.val, A.nnz * sizeof(double), k) != cudaSuccess) {
            free_batch(bt);
            return CBG_ERR_CUDA;
        }
        bool ok = rp[0] == 0 && rp[A.n] == A.nnz;
        for (long long i = 0; ok && i < A.n; i++) ok = rp[i + 1] >= rp[i];
        for (long long p = 0; ok && p < A.nnz; p++) ok = ci[p] >= 0 && ci[p] < A.n && std::isfinite(va[p]);
        if (!ok) { free_batch(bt); return CBG_ERR_ARG; }
        BatchSys d{};
        d.n = (int)A.n;
        d.ld = (int)((A.n + 63) / 64 * 64);
        d.rp_off = (long long)rp_all.size();
        d.nz_off = (long long)ci_all.size();
        d.vec_off = vec_off;
        d.v_off = v_off;
        d.pscale = 1.0;
        d.hscale = 1.0;
        v_off += (long long)(restart + 1) * d.ld * bs;
        v_off = (v_off + 255) / 256 * 256;
        vec_off += A.n;
        rp_all.insert(rp_all.end(), rp.begin(), rp.end());
        ci_all.insert(ci_all.end(), ci.begin(), ci.end());
        va_all.insert(va_all.end(), va.begin(), va.end());
        if (o.precond == CBG_PC_JACOBI) {
            std::vector<double> dinv(A.n, 0.0);
            for (long long i = 0; i < A.n; i++) {
                double dg = 0.0;
                for (int p = rp[i]; p < rp[i + 1]; p++)
                    if (ci[p] == i) dg = va[p];
                if (dg == 0.0) { free_batch(bt); return CBG_ERR_ARG; }
                dinv[i] = 1.0 / dg;
            }
            for (long long p = 0; p < A.nnz; p++) vp_all.push_back(va[p] * dinv[ci[p]]);
            di_all.insert(di_all.end(), dinv.begin(), dinv.end());
        }
        bt->sys.push_back(d);
        bt->total_rows += A.n;
        bt->total_nnz += A.nnz;
        bt->max_n = std::max(bt->max_n, (int)A.n);
    }
    bt->order.resize(nsys);
    std::iota(bt->order.begin(), bt->order.end(), 0);
    std::stable_sort(bt->order.begin(), bt->order.end(), [&](int a, int b) { return bt->sys[a].n > bt->sys[b].n; });
    auto up = [&](void** dst, const void* src, size_t bytes) -> int {
        if (cudaMalloc(dst, std::max<size_t>(bytes, 8)) != cudaSuccess) return CBG_ERR_OOM;
        if (bytes && cudaMemcpy(*dst, src, bytes, cudaMemcpyHostToDevice) != cudaSuccess) return CBG_ERR_CUDA;
        return CBG_OK;
    };
    int rc = CBG_OK;
    rc = rc ? rc : up((void**)&bt->d_order, bt->order.data(), bt->order.size() * sizeof(int));
    rc = rc ? rc : up((void**)&bt->d_rowptr, rp_all.data(), rp_all.size() * sizeof(int));
    rc = rc ? rc : up((void**)&bt->d_col, ci_all.data(), ci_all.size() * sizeof(int));
    rc = rc ? rc : up((void**)&bt->d_val, va_all.data(), va_all.size() * sizeof(double));
    if (o.precond == CBG_PC_JACOBI) {
        rc = rc ? rc : up((void**)&bt->d_valp, vp_all.data(), vp_all.size() * sizeof(double));
        rc = rc ? rc : up((void**)&bt->d_dinv, di_all.data(), di_all.size() * sizeof(double));
    }
    // each system's per-step operator normalised by a power of two (w = A v then stays near
    // unit size, far from FP32 underflow and overflow in the double-float sums; the
    // Hessenberg columns are scaled back exactly), and its values as double-float planes
    // unless some system's dynamic range exceeds 2^64 (FP64 products then)
    {
        const std::vector<double>& vs = o.precond == CBG_PC_JACOBI ? vp_all : va_all;
        bool df_ok = true;
        std::vector<int> ex(nsys);
        for (int i = 0; i < nsys; i++) {
            BatchSys& d = bt->sys[i];
            ex[i] = normalising_exponent(vs.data() + d.nz_off, As[i].nnz, df_ok);
            d.pscale = std::ldexp(1.0, ex[i]);
            d.hscale = std::ldexp(1.0, -ex[i]);
        }
        if (!rc && df_ok && fmt != CBG_F64) {       // (f64 codes keep FP64 products)
            std::vector<float> df(2 * vs.size());
            for (int i = 0; i < nsys; i++)
                split_values_df(vs.data() + bt->sys[i].nz_off, As[i].nnz, ex[i], df.data() + bt->sys[i].nz_off,
                                df.data() + vs.size() + bt->sys[i].nz_off);
            rc = up((void**)&bt->d_valpdf, df.data(), df.size() * sizeof(float));
        }
    }
    rc = rc ? rc : up((void**)&bt->d_sys, bt->sys.data(), bt->sys.size() * sizeof(BatchSys));
    if (!rc && cudaMalloc((void**)&bt->d_V, std::max<long long>(v_off, 256)) != cudaSuccess) rc = CBG_ERR_OOM;
    if (!rc && cudaMemset(bt->d_V, 0, std::max<long long>(v_off, 256)) != cudaSuccess) rc = CBG_ERR_CUDA;
    if (!rc && cudaMalloc((void**)&bt->d_out, nsys * sizeof(BatchOut)) != cudaSuccess) rc = CBG_ERR_OOM;
    if (!rc && cudaMalloc((void**)&bt->d_queue, 256) != cudaSuccess) rc = CBG_ERR_OOM;
    if (!rc && cudaMalloc((void**)&bt->d_io, 2 * sizeof(double*)) != cudaSuccess) rc = CBG_ERR_OOM;
    if (!rc && cudaHostAlloc((void**)&bt->h_io, 2 * sizeof(double*), cudaHostAllocDefault) != cudaSuccess) rc = CBG_ERR_OOM;
    if (!rc && (cudaEventCreate(&bt->e0) != cudaSuccess || cudaEventCreate(&bt->e1) != cudaSuccess)) rc = CBG_ERR_CUDA;
    if (!rc && cudaStreamCreateWithFlags(&bt->capture, cudaStreamNonBlocking) != cudaSuccess) rc = CBG_ERR_CUDA;
    if (rc) {
        free_batch(bt);
        return rc;
    }
    // default schedule: the largest cluster this GPU co-schedules (up to 8); systems of
    // 8192 rows or more on whole clusters
    Schedule sc;
    for (int c = 8; c >= 1; c /= 2) {
        Schedule t{c, c > 1 ? 8192 : (1 << 30)};
        if (grid_for(bt, t, smem_bytes(bt, t)) > 0) { sc = t; break; }
    }
    bt->sched = sc;
    *out = bt;
    return CBG_OK;
}

int cbgmres_solve_batched(cbg_batch* bt, const double* b, double* x, double tol, int64_t maxit, cbg_stats* per_sys)
{
    if (!bt || !b || !x || !(tol >= 0.0) || maxit < 0) return CBG_ERR_ARG;
    bt->h_io[0] = const_cast<double*>(b);
    bt->h_io[1] = x;
    const long long l0 = bt->launches;
    if (cudaEventRecord(bt->e0, bt->stream) != cudaSuccess) return CBG_ERR_CUDA;
    int rc;
    if (bt->opt.use_graph) {
        rc = run_graph(bt, tol, maxit);
    } else {
        const size_t sm = smem_bytes(bt, bt->sched);
        rc = enqueue(bt, bt->sched, grid_for(bt, bt->sched, sm), sm, tol, maxit, bt->stream);
    }
    if (rc) return rc;
    if (bt->opt.use_graph) bt->launches++;
    cudaError_t es = cudaEventRecord(bt->e1, bt->stream);
    if (es == cudaSuccess) es = cudaEventSynchronize(bt->e1);
    if (es == cudaSuccess) es = cudaGetLastError();
    if (es != cudaSuccess) { cbg_record_cuda_error(es); return CBG_ERR_CUDA; }
    float ms = 0.f;
    cudaEventElapsedTime(&ms, bt->e0, bt->e1);
    std::vector<BatchOut> o(bt->nsys);
    if (cudaMemcpy(o.data(), bt->d_out, bt->nsys * sizeof(BatchOut), cudaMemcpyDeviceToHost) != cudaSuccess)
        return CBG_ERR_CUDA;
    int worst = CBG_OK;
    for (int s = 0; s < bt->nsys; s++) {
        if (o[s].status < 0) worst = std::min(worst, o[s].status);
        else if (worst >= 0 && o[s].status > worst) worst = o[s].status;
        if (per_sys) {
            cbg_stats& st = per_sys[s];
            st.iters = o[s].iters;
            st.restarts = o[s].restarts;
            st.reorths = o[s].iters;
            st.true_relres = o[s].relres;
            st.est_relres = 0.0;
            st.ms_total = ms;
            st.bytes_model = 0.0;
            st.status = o[s].status;
            st.history_len = 0;
            st.kernel_launches = s == 0 ? bt->launches - l0 : 0;
        }
    }
    return worst;
}

// Time every candidate schedule on (b, x0) and keep the fastest.  x is restored to x0
// after every trial and holds the solution of the last trial on return.  cache_path
// (may be NULL): JSON-lines file consulted first and appended to.
int cbgmres_tune_batched(cbg_batch* bt, const double* b, double* x, double tol, int64_t maxit, const char* cache_path,
                         int* cluster_out, int* split_out)
{
    if (!bt || !b || !x) return CBG_ERR_ARG;
    const std::string key = tune_key(bt);
    Schedule best;
    if (cache_lookup(cache_path, key, &best) && grid_for(bt, best, smem_bytes(bt, best)) > 0) {
        bt->sched = best;
    } else {
        double* x0 = nullptr;
        if (cudaMalloc((void**)&x0, std::max<long long>(bt->total_rows, 1) * sizeof(double)) != cudaSuccess) return CBG_ERR_OOM;
        cudaMemcpyAsync(x0, x, bt->total_rows * sizeof(double), cudaMemcpyDeviceToDevice, bt->stream);
        std::vector<Schedule> cands;
        for (int c : {1, 2, 4, 8, 16})
            for (int sr : {2048, 4096, 8192, 16384, 32768}) {
                if (c == 1 && sr != 2048) continue;
                Schedule t{c, c == 1 ? (1 << 30) : sr};
                if (grid_for(bt, t, smem_bytes(bt, t)) > 0) cands.push_back(t);
            }
        double best_ms = 1e300;
        bt->h_io[0] = const_cast<double*>(b);
        bt->h_io[1] = x;
        auto trial = [&](const Schedule& t) {
            const size_t sm = smem_bytes(bt, t);
            const int grid = grid_for(bt, t, sm);
            cudaMemcpyAsync(x, x0, bt->total_rows * sizeof(double), cudaMemcpyDeviceToDevice, bt->stream);
            cudaEventRecord(bt->e0, bt->stream);
            int rc = enqueue(bt, t, grid, sm, tol, maxit, bt->stream);
            cudaEventRecord(bt->e1, bt->stream);
            if (rc || cudaEventSynchronize(bt->e1) != cudaSuccess) { cudaGetLastError(); return; }
            float ms = 0.f;
            cudaEventElapsedTime(&ms, bt->e0, bt->e1);
            if (ms < best_ms) { best_ms = ms; best = t; }
        };
        // cluster size and split threshold with a thread per SpMV row, then the SpMV's
        // lanes per row for the best of those
        for (const Schedule& t : cands) trial(t);
        const Schedule first = best;
        for (int l : {2, 4, 8}) {
            Schedule t = first;
            t.lanes = l;
            trial(t);
        }
        cudaFree(x0);
        if (best_ms >= 1e300) return CBG_ERR_CUDA;
        bt->sched = best;
        cache_store(cache_path, key, best, best_ms);
    }
    if (cluster_out) *cluster_out = bt->sched.cluster;
    if (split_out) *split_out = bt->sched.split_rows;
    return CBG_OK;
}

int cbgmres_batched_schedule(cbg_batch* bt, int cluster, int split_rows)
{
    if (!bt || cluster < 1 || cluster > 16 || (cluster & (cluster - 1)) || split_rows < 1) return CBG_ERR_ARG;
    Schedule t{cluster, split_rows, bt->sched.lanes};
    if (grid_for(bt, t, smem_bytes(bt, t)) <= 0) return CBG_ERR_UNSUPPORTED;
    bt->sched = t;
    return CBG_OK;
}

int cbgmres_batched_spmv_lanes(cbg_batch* bt, int lanes)
{
    if (!bt || lanes < 0 || lanes > 8 || (lanes & (lanes - 1))) return CBG_ERR_ARG;
    if (lanes > 0) bt->sched.lanes = lanes;
    return bt->sched.lanes;
}

void cbgmres_destroy_batched(cbg_batch* bt)
{
    if (bt) cudaStreamSynchronize(bt->stream);
    free_batch(bt);
}

}  // extern "C"
