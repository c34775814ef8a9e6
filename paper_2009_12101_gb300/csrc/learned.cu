// learned.cu -- learned sparse approximate inverse (SPAI) right preconditioner.
//
// A per-row MLP (7 stencil coefficients / a_ii -> 64 -> 64 -> 7, ReLU) emits the values
// of P on A's 7-point pattern: P_{i,nb(i,k)} = out_k(i) / a_ii.  The network is trained
// on (r, e) pairs with r = A e, e = x* - x_k from FP64 GMRES iterates, loss
//   L = mean over pairs of ||P r - e||^2 / ||e||^2.
// L is quadratic in each row's seven P values, so the pairs enter only through per-row
// statistics G_i = sum w r_nb r_nb^T (7x7), c_i = sum w e_i r_nb, d_i = sum w e_i^2
// (w = 1/||e||^2), accumulated on the GPU as pairs arrive; every training step is then
// one fused pass of the network over the rows on the tensor cores (mlp_tc.cu: forward,
// loss, backward, weight gradients), the cross-CTA gradient sum in FP64 and an Adam
// update of the FP32 master weights, which the network uses rounded to BF16.
// The paper has no learned preconditioner; it composes with any preconditioner.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <random>
#include <vector>

#include "../../include/cbgmres.h"
#include "cbg_device.cuh"
#include "cbg_mlp.h"

using namespace cbg;

void cbg_record_cuda_error(cudaError_t e);   // solver.cu

namespace {

constexpr int LT = 256;            // threads of the row kernels

__global__ void k_spai_setup(const int* rowptr, const int* col, const double* val, long long n, long long sx,
                             long long sxy, signed char* slot, float* feat, double* diag, unsigned char* mask,
                             int* bad)
{
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const long long off[7] = {-sxy, -sx, -1, 0, 1, sx, sxy};
        double a[7] = {0, 0, 0, 0, 0, 0, 0};
        unsigned char m = 0;
        for (int p = rowptr[i]; p < rowptr[i + 1]; p++) {
            const long long dl = (long long)col[p] - i;
            int k = -1;
            for (int t = 0; t < 7; t++)
                if (off[t] == dl) k = t;
            if (k < 0 || (m >> k) & 1) { atomicExch(bad, 1); k = 3; }
            slot[p] = (signed char)k;
            a[k] = val[p];
            m |= (unsigned char)(1u << k);
        }
        const double d = a[3];
        if (!(d != 0.0) || !isfinite(d)) atomicExch(bad, 1);
        diag[i] = d;
        mask[i] = m;
        for (int k = 0; k < 7; k++) feat[i * 7 + k] = (float)(a[k] / d);
    }
}

// r = A e (e = x* - x_k formed on the fly), and ||e||^2 per block
__global__ void k_pair_residual(const int* rowptr, const int* col, const double* val, long long n,
                                const double* xs, const double* xk, double* e, double* r, double* part)
{
    __shared__ double red[LT / 32];
    double ss = 0.0;
    for (long long i = (long long)blockIdx.x * LT + threadIdx.x; i < n; i += (long long)gridDim.x * LT) {
        double t = 0.0;
        for (int p = rowptr[i]; p < rowptr[i + 1]; p++) {
            const int c = col[p];
            t = __fma_rn(val[p], __dsub_rn(xs[c], xk[c]), t);
        }
        const double ei = __dsub_rn(xs[i], xk[i]);
        e[i] = ei;
        r[i] = t;
        ss = __fma_rn(ei, ei, ss);
    }
    ss = warp_sum(ss);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = ss;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < LT / 32; w++) t += red[w];
        part[blockIdx.x] = t;
    }
}

// add one pair (weight 1/||e||^2, from the block partials) to G, c, d
__global__ void k_pair_accumulate(const int* rowptr, const int* col, const signed char* slot, long long n,
                                  const double* r, const double* e, const double* part, int nparts, float* G,
                                  float* c, float* d)
{
    __shared__ double wgt;
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int b = 0; b < nparts; b++) t += part[b];
        wgt = t > 0.0 ? 1.0 / t : 0.0;
    }
    __syncthreads();
    const float w = (float)wgt;
    for (long long i = (long long)blockIdx.x * LT + threadIdx.x; i < n; i += (long long)gridDim.x * LT) {
        float rv[7] = {0, 0, 0, 0, 0, 0, 0};
        for (int p = rowptr[i]; p < rowptr[i + 1]; p++) rv[slot[p]] = (float)r[col[p]];
        const float ei = (float)e[i];
        for (int k = 0; k < 7; k++) {
            const float wr = w * rv[k];
            for (int l = 0; l < 7; l++) G[i * 49 + k * 7 + l] += wr * rv[l];
            c[i * 7 + k] += wr * ei;
        }
        d[i] += w * ei * ei;
    }
}

// grad[idx] = sum over the CTAs' partials gpart[b][idx] in FP64.  Block x covers the 32
// parameters 32x .. 32x+31 (one per lane, coalesced rows of gpart); its eight warps take
// the partials b = w, w + 8, ... (eight loads in flight per lane), and the warps' sums are
// added in warp order: a fixed order for a given nblk.
constexpr int GR_THREADS = 256;
__global__ void __launch_bounds__(GR_THREADS) k_grad_reduce(const float* gpart, int nblk, double* grad)
{
    __shared__ double part[GR_THREADS / 32][32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int idx = blockIdx.x * 32 + lane;
    double t = 0.0;
    if (idx < NPARAM) {
        for (int b0 = warp; b0 < nblk; b0 += 8 * (GR_THREADS / 32)) {
            float v[8];
#pragma unroll
            for (int u = 0; u < 8; u++) {
                const int b = b0 + u * (GR_THREADS / 32);
                v[u] = b < nblk ? gpart[(long long)b * NPARAM + idx] : 0.f;
            }
#pragma unroll
            for (int u = 0; u < 8; u++)
                if (b0 + u * (GR_THREADS / 32) < nblk) t = __dadd_rn(t, f32_to_f64_exact(v[u]));
        }
    }
    part[warp][lane] = t;
    __syncthreads();
    if (warp == 0 && idx < NPARAM) {
        double s = 0.0;
#pragma unroll
        for (int w = 0; w < GR_THREADS / 32; w++) s = __dadd_rn(s, part[w][lane]);
        grad[idx] = s;
    }
}

// Adam on the FP32 master weights; the BF16-rounded copy is what the network computes with
__global__ void k_adam(float* master, float* bf, const double* grad, float* m1, float* m2, int step, float lr,
                       float b1, float b2, float eps)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < NPARAM; i += gridDim.x * blockDim.x) {
        const float g = (float)grad[i];
        const float a = b1 * m1[i] + (1.f - b1) * g;
        const float v = b2 * m2[i] + (1.f - b2) * g * g;
        m1[i] = a;
        m2[i] = v;
        const float ah = a / (1.f - powf(b1, (float)step));
        const float vh = v / (1.f - powf(b2, (float)step));
        const float w = master[i] - lr * ah / (sqrtf(vh) + eps);
        master[i] = w;
        bf[i] = __bfloat162float(__float2bfloat16_rn(w));
    }
}

__global__ void k_round_bf16(const float* master, float* bf)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < NPARAM; i += gridDim.x * blockDim.x)
        bf[i] = __bfloat162float(__float2bfloat16_rn(master[i]));
}

__global__ void k_spai_pvals(const int* rowptr, const signed char* slot, long long n, const float* out,
                             const double* diag, double* pvals)
{
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const double id = 1.0 / diag[i];
        for (int p = rowptr[i]; p < rowptr[i + 1]; p++) pvals[p] = (double)out[i * 7 + slot[p]] * id;
    }
}

int grid_rows(long long n) { return (int)std::max<long long>(1, std::min<long long>((n + LT - 1) / LT, 4096)); }

}  // namespace

struct cbg_spai {
    long long n = 0, nnz = 0;
    cudaStream_t stream = nullptr;
    int *rowptr = nullptr, *col = nullptr;
    double* val = nullptr;
    signed char* slot = nullptr;
    unsigned char* mask = nullptr;
    float* feat = nullptr;
    double* diag = nullptr;
    float *G = nullptr, *c = nullptr, *d = nullptr;
    double *e = nullptr, *r = nullptr, *part = nullptr;
    float *master = nullptr, *bf = nullptr, *m1 = nullptr, *m2 = nullptr, *out = nullptr;
    float* gpart = nullptr;       // per-CTA gradient partials of the network kernel
    double* lpart = nullptr;      // per-CTA loss partials
    double* grad = nullptr;
    int* fault = nullptr;         // a tensor-core wait ran out
    int tc_grid = 0;
    long long npairs = 0;
    int step = 0;
};

namespace {

void free_spai(cbg_spai* s)
{
    if (!s) return;
    void* ps[] = {s->rowptr, s->col, s->val, s->slot, s->mask, s->feat, s->diag, s->G, s->c, s->d, s->e, s->r,
                  s->part, s->master, s->bf, s->m1, s->m2, s->out, s->gpart, s->lpart, s->grad, s->fault};
    for (void* p : ps) cudaFree(p);
    delete s;
}

template <class T> int alloc(T** p, size_t count)
{
    cudaError_t e = cudaMalloc((void**)p, std::max<size_t>(count, 1) * sizeof(T));
    if (e != cudaSuccess) {
        *p = nullptr;
        cbg_record_cuda_error(e);
        return e == cudaErrorMemoryAllocation ? CBG_ERR_OOM : CBG_ERR_CUDA;
    }
    return CBG_OK;
}

int check(cudaError_t e)
{
    if (e != cudaSuccess) {
        cbg_record_cuda_error(e);
        return CBG_ERR_CUDA;
    }
    return CBG_OK;
}

// deterministic initialisation: He-scaled uniform weights from a fixed-seed generator,
// output layer small with b3 = e_centre, so the first P is the Jacobi preconditioner
void init_params(std::vector<float>& w, unsigned long long seed)
{
    std::mt19937_64 g(seed);
    std::uniform_real_distribution<float> u(-1.f, 1.f);
    w.assign(NPARAM, 0.f);
    for (int i = 0; i < NH * NIN; i++) w[OFF_W1 + i] = u(g) * std::sqrt(6.f / NIN);
    for (int i = 0; i < NH; i++) w[OFF_B1 + i] = 0.1f * u(g);
    for (int i = 0; i < NH * NH; i++) w[OFF_W2 + i] = u(g) * std::sqrt(6.f / NH);
    for (int i = 0; i < NH; i++) w[OFF_B2 + i] = 0.1f * u(g);
    for (int i = 0; i < NOUT * NH; i++) w[OFF_W3 + i] = 1e-3f * u(g);
    w[OFF_B3 + 3] = 1.f;
}

MlpArgs net_args(const cbg_spai* s)
{
    MlpArgs a{};
    a.n = s->n;
    a.feat = s->feat;
    a.params = s->bf;
    a.G = s->G;
    a.c = s->c;
    a.d = s->d;
    a.diag = s->diag;
    a.mask = s->mask;
    a.inv_npairs = 1.0 / (double)std::max<long long>(1, s->npairs);
    a.gpart = s->gpart;
    a.lpart = s->lpart;
    a.fault = s->fault;
    return a;
}

// one fused pass of the network on the tensor cores: loss partials and the weight
// gradient's per-CTA partials; with `loss`, the loss is read back (synchronising)
int train_pass(cbg_spai* s, double* loss)
{
    int rc = check(mlp_tc_launch(MLP_TRAIN, s->tc_grid, s->stream, net_args(s)));
    if (rc || !loss) return rc;
    std::vector<double> parts(s->tc_grid);
    int fault = 0;
    rc = check(cudaMemcpyAsync(parts.data(), s->lpart, s->tc_grid * sizeof(double), cudaMemcpyDeviceToHost, s->stream));
    if (!rc) rc = check(cudaMemcpyAsync(&fault, s->fault, sizeof(int), cudaMemcpyDeviceToHost, s->stream));
    if (!rc) rc = check(cudaStreamSynchronize(s->stream));
    if (rc) return rc;
    if (fault) return CBG_ERR_TIMEOUT;
    double t = 0.0;
    for (double v : parts) t += v;
    *loss = t;
    return CBG_OK;
}

}  // namespace

extern "C" {

int cbg_spai_create(const cbg_csr* A, int64_t sx, int64_t sxy, const cbg_options* opt, cbg_spai** out)
{
    if (!out) return CBG_ERR_ARG;
    *out = nullptr;
    if (!A || A->n < 1 || A->nnz < 1 || !A->row_ptr || !A->col || !A->val || sx < 1 || sxy < sx) return CBG_ERR_ARG;
    cbg_spai* s = new (std::nothrow) cbg_spai();
    if (!s) return CBG_ERR_OOM;
    s->n = A->n;
    s->nnz = A->nnz;
    s->stream = opt ? (cudaStream_t)opt->stream : nullptr;
    const long long n = s->n, nnz = s->nnz;
    int rc = CBG_OK;
#define TRY(x)                 \
    do {                       \
        rc = (x);              \
        if (rc) {              \
            free_spai(s);      \
            return rc;         \
        }                      \
    } while (0)
    // per-row arrays of the network are padded to whole 128-row tiles (padding rows zero,
    // diagonal one), so the tensor-core kernel stages full tiles
    const long long np = (n + MLP_ROWS - 1) / MLP_ROWS * MLP_ROWS;
    TRY(alloc(&s->rowptr, n + 1)); TRY(alloc(&s->col, nnz)); TRY(alloc(&s->val, nnz));
    const cudaMemcpyKind k = A->on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    TRY(check(cudaMemcpy(s->rowptr, A->row_ptr, (n + 1) * sizeof(int), k)));
    TRY(check(cudaMemcpy(s->col, A->col, nnz * sizeof(int), k)));
    TRY(check(cudaMemcpy(s->val, A->val, nnz * sizeof(double), k)));
    TRY(alloc(&s->slot, nnz)); TRY(alloc(&s->mask, np)); TRY(alloc(&s->feat, np * NIN)); TRY(alloc(&s->diag, np));
    TRY(alloc(&s->G, np * 49)); TRY(alloc(&s->c, np * 7)); TRY(alloc(&s->d, np));
    TRY(alloc(&s->e, n)); TRY(alloc(&s->r, n)); TRY(alloc(&s->part, 4096));
    TRY(alloc(&s->master, NPARAM)); TRY(alloc(&s->bf, NPARAM)); TRY(alloc(&s->m1, NPARAM)); TRY(alloc(&s->m2, NPARAM));
    TRY(alloc(&s->out, np * NOUT)); TRY(alloc(&s->grad, NPARAM)); TRY(alloc(&s->fault, 1));
    s->tc_grid = mlp_tc_grid(n);
    TRY(alloc(&s->gpart, (size_t)s->tc_grid * NPARAM));
    TRY(alloc(&s->lpart, (size_t)s->tc_grid));
    TRY(check(cudaMemset(s->G, 0, np * 49 * sizeof(float))));
    TRY(check(cudaMemset(s->c, 0, np * 7 * sizeof(float))));
    TRY(check(cudaMemset(s->d, 0, np * sizeof(float))));
    TRY(check(cudaMemset(s->mask, 0, np)));
    TRY(check(cudaMemset(s->feat, 0, np * NIN * sizeof(float))));
    TRY(check(cudaMemset(s->fault, 0, sizeof(int))));
    if (np > n) {
        std::vector<double> ones(np - n, 1.0);
        TRY(check(cudaMemcpy(s->diag + n, ones.data(), (np - n) * sizeof(double), cudaMemcpyHostToDevice)));
    }
    TRY(check(cudaMemset(s->m1, 0, NPARAM * sizeof(float))));
    TRY(check(cudaMemset(s->m2, 0, NPARAM * sizeof(float))));
    int* bad = reinterpret_cast<int*>(s->part);
    TRY(check(cudaMemset(bad, 0, sizeof(int))));
    k_spai_setup<<<grid_rows(n), LT>>>(s->rowptr, s->col, s->val, n, sx, sxy, s->slot, s->feat, s->diag, s->mask, bad);
    int hbad = 0;
    TRY(check(cudaMemcpy(&hbad, bad, sizeof(int), cudaMemcpyDeviceToHost)));
    if (hbad) TRY(CBG_ERR_ARG);   // not a 7-point pattern with these strides, or a zero diagonal
    std::vector<float> w;
    init_params(w, 20201201ull);
    TRY(check(cudaMemcpy(s->master, w.data(), NPARAM * sizeof(float), cudaMemcpyHostToDevice)));
    k_round_bf16<<<32, 256>>>(s->master, s->bf);
    TRY(check(cudaDeviceSynchronize()));
#undef TRY
    *out = s;
    return CBG_OK;
}

int cbg_spai_add_pair(cbg_spai* s, const double* xstar, const double* xk)
{
    if (!s || !xstar || !xk) return CBG_ERR_ARG;
    const int g = grid_rows(s->n);
    k_pair_residual<<<g, LT, 0, s->stream>>>(s->rowptr, s->col, s->val, s->n, xstar, xk, s->e, s->r, s->part);
    k_pair_accumulate<<<g, LT, 0, s->stream>>>(s->rowptr, s->col, s->slot, s->n, s->r, s->e, s->part, g, s->G, s->c,
                                              s->d);
    int rc = check(cudaGetLastError());
    if (!rc) s->npairs++;
    return rc;
}

int cbg_spai_loss(cbg_spai* s, double* loss)
{
    if (!s || !loss || s->npairs < 1) return CBG_ERR_ARG;
    return train_pass(s, loss);
}

int cbg_spai_train(cbg_spai* s, int steps, double lr, double* loss_first, double* loss_last)
{
    if (!s || steps < 0 || !(lr > 0.0) || s->npairs < 1) return CBG_ERR_ARG;
    double l0 = 0.0, l = 0.0;
    for (int it = 0; it < steps; it++) {
        // the loss is read back once, before the first update (no per-step synchronisation)
        int rc = train_pass(s, it == 0 ? &l0 : nullptr);
        if (rc) return rc;
        k_grad_reduce<<<(NPARAM + 31) / 32, GR_THREADS, 0, s->stream>>>(s->gpart, s->tc_grid, s->grad);
        s->step++;
        k_adam<<<(NPARAM + 255) / 256, 256, 0, s->stream>>>(s->master, s->bf, s->grad, s->m1, s->m2, s->step,
                                                            (float)lr, 0.9f, 0.999f, 1e-8f);
        rc = check(cudaGetLastError());
        if (rc) return rc;
    }
    int rc = train_pass(s, &l);                           // the loss after the last update
    if (rc) return rc;
    if (steps == 0) l0 = l;
    if (loss_first) *loss_first = l0;
    if (loss_last) *loss_last = l;
    return CBG_OK;
}

int cbg_spai_values(cbg_spai* s, double* pvals)
{
    if (!s || !pvals) return CBG_ERR_ARG;
    const int g = grid_rows(s->n);
    MlpArgs a = net_args(s);
    a.out = s->out;
    int rc = check(mlp_tc_launch(MLP_FWD, s->tc_grid, s->stream, a));
    if (rc) return rc;
    k_spai_pvals<<<g, LT, 0, s->stream>>>(s->rowptr, s->slot, s->n, s->out, s->diag, pvals);
    rc = check(cudaGetLastError());
    if (!rc) rc = check(cudaStreamSynchronize(s->stream));
    return rc;
}

int cbg_spai_params(cbg_spai* s, float* params, int set)
{
    if (!s || !params) return CBG_ERR_ARG;
    if (set) {
        int rc = check(cudaMemcpy(s->master, params, NPARAM * sizeof(float), cudaMemcpyHostToDevice));
        if (rc) return rc;
        k_round_bf16<<<32, 256, 0, s->stream>>>(s->master, s->bf);
        return check(cudaStreamSynchronize(s->stream));
    }
    return check(cudaMemcpy(params, s->master, NPARAM * sizeof(float), cudaMemcpyDeviceToHost));
}

int cbg_spai_num_params(void) { return NPARAM; }

void cbg_spai_destroy(cbg_spai* s)
{
    if (s) cudaStreamSynchronize(s->stream);
    free_spai(s);
}

// ---- test access: one forward / backward with given FP32 parameters (rounded to BF16),
// on the tensor-core kernel
int cbg_mlp_forward(int64_t rows, const float* feat, const float* params_host, float* out, void* stream)
{
    if (rows < 1 || !feat || !params_host || !out || ((uintptr_t)feat & 15)) return CBG_ERR_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    float *m = nullptr, *b = nullptr;
    int* fault = nullptr;
    int rc = alloc(&m, NPARAM);
    if (!rc) rc = alloc(&b, NPARAM);
    if (!rc) rc = alloc(&fault, 1);
    if (!rc) rc = check(cudaMemsetAsync(fault, 0, sizeof(int), st));
    if (!rc) rc = check(cudaMemcpyAsync(m, params_host, NPARAM * sizeof(float), cudaMemcpyHostToDevice, st));
    if (!rc) {
        k_round_bf16<<<32, 256, 0, st>>>(m, b);
        MlpArgs a{};
        a.n = rows;
        a.feat = feat;
        a.params = b;
        a.out = out;
        a.fault = fault;
        rc = check(mlp_tc_launch(MLP_FWD, mlp_tc_grid(rows), st, a));
        int hf = 0;
        if (!rc) rc = check(cudaMemcpyAsync(&hf, fault, sizeof(int), cudaMemcpyDeviceToHost, st));
        if (!rc) rc = check(cudaStreamSynchronize(st));
        if (!rc && hf) rc = CBG_ERR_TIMEOUT;
    }
    cudaFree(m);
    cudaFree(b);
    cudaFree(fault);
    return rc;
}

int cbg_mlp_backward(int64_t rows, const float* feat, const float* params_host, const float* gout, double* grad_host,
                     void* stream)
{
    if (rows < 1 || !feat || !params_host || !gout || !grad_host || ((uintptr_t)feat & 15) || ((uintptr_t)gout & 15))
        return CBG_ERR_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    const int grid = mlp_tc_grid(rows);
    float *m = nullptr, *b = nullptr, *gp = nullptr;
    double* g = nullptr;
    int* fault = nullptr;
    int rc = alloc(&m, NPARAM);
    if (!rc) rc = alloc(&b, NPARAM);
    if (!rc) rc = alloc(&gp, (size_t)grid * NPARAM);
    if (!rc) rc = alloc(&g, NPARAM);
    if (!rc) rc = alloc(&fault, 1);
    if (!rc) rc = check(cudaMemsetAsync(fault, 0, sizeof(int), st));
    if (!rc) rc = check(cudaMemcpyAsync(m, params_host, NPARAM * sizeof(float), cudaMemcpyHostToDevice, st));
    if (!rc) {
        k_round_bf16<<<32, 256, 0, st>>>(m, b);
        MlpArgs a{};
        a.n = rows;
        a.feat = feat;
        a.params = b;
        a.gout = gout;
        a.gpart = gp;
        a.fault = fault;
        rc = check(mlp_tc_launch(MLP_BWD, grid, st, a));
        if (!rc) {
            k_grad_reduce<<<(NPARAM + 31) / 32, GR_THREADS, 0, st>>>(gp, grid, g);
            rc = check(cudaGetLastError());
        }
        int hf = 0;
        if (!rc) rc = check(cudaMemcpyAsync(grad_host, g, NPARAM * sizeof(double), cudaMemcpyDeviceToHost, st));
        if (!rc) rc = check(cudaMemcpyAsync(&hf, fault, sizeof(int), cudaMemcpyDeviceToHost, st));
        if (!rc) rc = check(cudaStreamSynchronize(st));
        if (!rc && hf) rc = CBG_ERR_TIMEOUT;
    }
    cudaFree(m); cudaFree(b); cudaFree(gp); cudaFree(g); cudaFree(fault);
    return rc;
}

}  // extern "C"
