// learned.cu -- learned sparse approximate inverse (SPAI) right preconditioner.
//
// A per-row MLP (7 stencil coefficients / a_ii -> 64 -> 64 -> 7, ReLU) emits the values
// of P on A's 7-point pattern: P_{i,nb(i,k)} = out_k(i) / a_ii.  The network is trained
// on (r, e) pairs with r = A e, e = x* - x_k from FP64 GMRES iterates, loss
//   L = mean over pairs of ||P r - e||^2 / ||e||^2.
// L is quadratic in each row's seven P values, so the pairs enter only through per-row
// statistics G_i = sum w r_nb r_nb^T (7x7), c_i = sum w e_i r_nb, d_i = sum w e_i^2
// (w = 1/||e||^2), accumulated on the GPU as pairs arrive; every training step is then
// one MLP forward and backward over the rows.  Weights are BF16 values (FP32 master copy
// updated by Adam), all sums accumulate in FP32, the cross-block gradient sum in FP64.
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

using namespace cbg;

void cbg_record_cuda_error(cudaError_t e);   // solver.cu

namespace {

constexpr int NIN = 7, NH = 64, NOUT = 7;
constexpr int OFF_W1 = 0, OFF_B1 = OFF_W1 + NH * NIN, OFF_W2 = OFF_B1 + NH, OFF_B2 = OFF_W2 + NH * NH,
              OFF_W3 = OFF_B2 + NH, OFF_B3 = OFF_W3 + NOUT * NH, NPARAM = OFF_B3 + NOUT;   // 5127
constexpr int LT = 256;            // threads of the row kernels
constexpr int BT = 128;            // rows per tile of the backward kernel

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

// -------------------------------------------------------------------- MLP forward
__device__ __forceinline__ void load_params(const float* __restrict__ P, float* s)
{
    for (int i = threadIdx.x; i < NPARAM; i += blockDim.x) s[i] = P[i];
    __syncthreads();
}

__global__ void __launch_bounds__(LT) k_mlp_forward(long long n, const float* __restrict__ feat,
                                                    const float* __restrict__ params, float* __restrict__ out)
{
    __shared__ float sp[NPARAM];
    load_params(params, sp);
    for (long long i = (long long)blockIdx.x * LT + threadIdx.x; i < n; i += (long long)gridDim.x * LT) {
        float f[NIN];
#pragma unroll
        for (int k = 0; k < NIN; k++) f[k] = feat[i * NIN + k];
        float h1[NH];
#pragma unroll
        for (int o = 0; o < NH; o++) {
            float z = sp[OFF_B1 + o];
#pragma unroll
            for (int k = 0; k < NIN; k++) z = fmaf(sp[OFF_W1 + o * NIN + k], f[k], z);
            h1[o] = fmaxf(z, 0.f);
        }
        float y[NOUT];
#pragma unroll
        for (int k = 0; k < NOUT; k++) y[k] = sp[OFF_B3 + k];
        for (int o = 0; o < NH; o++) {
            float z = sp[OFF_B2 + o];
#pragma unroll
            for (int q = 0; q < NH; q++) z = fmaf(sp[OFF_W2 + o * NH + q], h1[q], z);
            const float h2 = fmaxf(z, 0.f);
#pragma unroll
            for (int k = 0; k < NOUT; k++) y[k] = fmaf(sp[OFF_W3 + k * NH + o], h2, y[k]);
        }
#pragma unroll
        for (int k = 0; k < NOUT; k++) out[i * NOUT + k] = y[k];
    }
}

// loss and dL/dout from the per-row statistics
__global__ void k_spai_loss(long long n, const float* __restrict__ out, const float* __restrict__ G,
                            const float* __restrict__ c, const float* __restrict__ d, const double* __restrict__ diag,
                            const unsigned char* __restrict__ mask, double inv_npairs, float* __restrict__ gout,
                            double* __restrict__ part)
{
    __shared__ double red[LT / 32];
    double ls = 0.0;
    for (long long i = (long long)blockIdx.x * LT + threadIdx.x; i < n; i += (long long)gridDim.x * LT) {
        const float id = (float)(1.0 / diag[i]);
        const unsigned char m = mask[i];
        float p[7];
#pragma unroll
        for (int k = 0; k < 7; k++) p[k] = (m >> k) & 1 ? out[i * 7 + k] * id : 0.f;
        float li = d[i];
#pragma unroll
        for (int k = 0; k < 7; k++) {
            float gp = 0.f;
#pragma unroll
            for (int l = 0; l < 7; l++) gp = fmaf(G[i * 49 + k * 7 + l], p[l], gp);
            const float ck = c[i * 7 + k];
            li = fmaf(p[k], gp - 2.f * ck, li);
            if (gout) gout[i * 7 + k] = (m >> k) & 1 ? 2.f * (gp - ck) * id * (float)inv_npairs : 0.f;
        }
        ls += (double)li;
    }
    ls = warp_sum(ls);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = ls;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < LT / 32; w++) t += red[w];
        part[blockIdx.x] = t * inv_npairs;
    }
}

// -------------------------------------------------------------------- MLP backward
// Tiles of BT rows: phase 1 (TPR threads per row, each an equal share of the hidden
// units) recomputes the forward pass and writes
// H1, H2, D2 = relu'(z2) * (W3^T gout), D1 = relu'(z1) * (W2^T D2) to shared memory;
// phase 2 (all threads) accumulates the weight gradients as small dense products over
// the tile (gW2 = D2^T H1, gW1 = D1^T F, gW3 = Gout^T H2, bias = column sums) in
// registers; each block writes its partial gradient, a second kernel adds them in FP64.
struct BwdSmem {
    float p[NPARAM];
    float H1[BT][NH + 1];
    float H2[BT][NH + 1];
    float D1[BT][NH + 1];
    float D2[BT][NH + 1];
    float F[BT][NIN];
    float Go[BT][NOUT];
};

constexpr int BWD_THREADS = 512;
constexpr int TPR = BWD_THREADS / BT;                            // threads per row in the row phase
static_assert(BWD_THREADS == TPR * BT && NH % TPR == 0, "the row phase splits the hidden units evenly");
constexpr int GPT = (NPARAM + BWD_THREADS - 1) / BWD_THREADS;   // gradient entries per thread (11)

__global__ void __launch_bounds__(BWD_THREADS) k_mlp_backward(long long n, const float* __restrict__ feat,
                                                              const float* __restrict__ params,
                                                              const float* __restrict__ gout, float* __restrict__ gpart)
{
    extern __shared__ __align__(16) unsigned char bwd_raw[];
    BwdSmem& s = *reinterpret_cast<BwdSmem*>(bwd_raw);
    load_params(params, s.p);
    float acc[GPT];
#pragma unroll
    for (int q = 0; q < GPT; q++) acc[q] = 0.f;
    const long long ntiles = (n + BT - 1) / BT;
    for (long long t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const long long i0 = t * BT;
        __syncthreads();
        // TPR threads per row, each taking an equal share of the hidden units of every
        // layer (the same operations in the same order as one thread per row, so the
        // same values)
        {
            const int rr = threadIdx.x % BT, hf = threadIdx.x / BT;
            const int u0 = hf * (NH / TPR), u1 = u0 + NH / TPR;
            const long long i = i0 + rr;
            const bool valid = i < n;
            float f[NIN], g[NOUT];
#pragma unroll
            for (int k = 0; k < NIN; k++) f[k] = valid ? feat[i * NIN + k] : 0.f;
#pragma unroll
            for (int k = 0; k < NOUT; k++) g[k] = valid ? gout[i * NOUT + k] : 0.f;
            if (hf == 0) {
#pragma unroll
                for (int k = 0; k < NIN; k++) s.F[rr][k] = f[k];
#pragma unroll
                for (int k = 0; k < NOUT; k++) s.Go[rr][k] = g[k];
            }
            for (int o = u0; o < u1; o++) {
                float z = s.p[OFF_B1 + o];
#pragma unroll
                for (int k = 0; k < NIN; k++) z = fmaf(s.p[OFF_W1 + o * NIN + k], f[k], z);
                s.H1[rr][o] = valid ? fmaxf(z, 0.f) : 0.f;
            }
            __syncthreads();                                     // the row's whole H1
            for (int o = u0; o < u1; o++) {
                float z = s.p[OFF_B2 + o];
                for (int q = 0; q < NH; q++) z = fmaf(s.p[OFF_W2 + o * NH + q], s.H1[rr][q], z);
                float dz = 0.f;
#pragma unroll
                for (int k = 0; k < NOUT; k++) dz = fmaf(s.p[OFF_W3 + k * NH + o], g[k], dz);
                s.H2[rr][o] = valid ? fmaxf(z, 0.f) : 0.f;
                s.D2[rr][o] = (valid && z > 0.f) ? dz : 0.f;
            }
            __syncthreads();                                     // the row's whole D2
            for (int q = u0; q < u1; q++) {
                float dz = 0.f;
                for (int o = 0; o < NH; o++) dz = fmaf(s.p[OFF_W2 + o * NH + q], s.D2[rr][o], dz);
                s.D1[rr][q] = s.H1[rr][q] > 0.f ? dz : 0.f;
            }
        }
        __syncthreads();
        const int rows = (int)(n - i0 < BT ? n - i0 : BT);
#pragma unroll
        for (int q = 0; q < GPT; q++) {
            const int idx = threadIdx.x + q * BWD_THREADS;
            if (idx >= NPARAM) break;
            float a = 0.f;
            if (idx < OFF_B1) {                                  // W1[o][k] += D1[r][o] F[r][k]
                const int o = idx / NIN, k = idx % NIN;
                for (int r = 0; r < rows; r++) a = fmaf(s.D1[r][o], s.F[r][k], a);
            } else if (idx < OFF_W2) {                           // b1
                const int o = idx - OFF_B1;
                for (int r = 0; r < rows; r++) a += s.D1[r][o];
            } else if (idx < OFF_B2) {                           // W2[o][q] += D2[r][o] H1[r][q]
                const int o = (idx - OFF_W2) / NH, qq = (idx - OFF_W2) % NH;
                for (int r = 0; r < rows; r++) a = fmaf(s.D2[r][o], s.H1[r][qq], a);
            } else if (idx < OFF_W3) {                           // b2
                const int o = idx - OFF_B2;
                for (int r = 0; r < rows; r++) a += s.D2[r][o];
            } else if (idx < OFF_B3) {                           // W3[k][o] += Go[r][k] H2[r][o]
                const int k = (idx - OFF_W3) / NH, o = (idx - OFF_W3) % NH;
                for (int r = 0; r < rows; r++) a = fmaf(s.Go[r][k], s.H2[r][o], a);
            } else {                                             // b3
                const int k = idx - OFF_B3;
                for (int r = 0; r < rows; r++) a += s.Go[r][k];
            }
            acc[q] += a;
        }
    }
#pragma unroll
    for (int q = 0; q < GPT; q++) {
        const int idx = threadIdx.x + q * BWD_THREADS;
        if (idx < NPARAM) gpart[(long long)blockIdx.x * NPARAM + idx] = acc[q];
    }
}

__global__ void k_grad_reduce(const float* gpart, int nblk, double* grad)
{
    for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < NPARAM; idx += gridDim.x * blockDim.x) {
        double t = 0.0;
        for (int b = 0; b < nblk; b++) t += (double)gpart[(long long)b * NPARAM + idx];
        grad[idx] = t;
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
    float *master = nullptr, *bf = nullptr, *m1 = nullptr, *m2 = nullptr, *out = nullptr, *gout = nullptr;
    float* gpart = nullptr;
    double* grad = nullptr;
    int bwd_grid = 0;
    long long npairs = 0;
    int step = 0;
};

namespace {

void free_spai(cbg_spai* s)
{
    if (!s) return;
    void* ps[] = {s->rowptr, s->col, s->val, s->slot, s->mask, s->feat, s->diag, s->G, s->c, s->d, s->e, s->r,
                  s->part, s->master, s->bf, s->m1, s->m2, s->out, s->gout, s->gpart, s->grad};
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

int forward_and_loss(cbg_spai* s, double* loss, bool want_grad)
{
    const int g = grid_rows(s->n);
    k_mlp_forward<<<g, LT, 0, s->stream>>>(s->n, s->feat, s->bf, s->out);
    k_spai_loss<<<g, LT, 0, s->stream>>>(s->n, s->out, s->G, s->c, s->d, s->diag, s->mask,
                                         1.0 / (double)std::max<long long>(1, s->npairs), want_grad ? s->gout : nullptr,
                                         s->part);
    std::vector<double> parts(g);
    int rc = check(cudaMemcpyAsync(parts.data(), s->part, g * sizeof(double), cudaMemcpyDeviceToHost, s->stream));
    if (!rc) rc = check(cudaStreamSynchronize(s->stream));
    if (rc) return rc;
    double t = 0.0;
    for (double v : parts) t += v;
    if (loss) *loss = t;
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
    TRY(alloc(&s->rowptr, n + 1)); TRY(alloc(&s->col, nnz)); TRY(alloc(&s->val, nnz));
    const cudaMemcpyKind k = A->on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    TRY(check(cudaMemcpy(s->rowptr, A->row_ptr, (n + 1) * sizeof(int), k)));
    TRY(check(cudaMemcpy(s->col, A->col, nnz * sizeof(int), k)));
    TRY(check(cudaMemcpy(s->val, A->val, nnz * sizeof(double), k)));
    TRY(alloc(&s->slot, nnz)); TRY(alloc(&s->mask, n)); TRY(alloc(&s->feat, n * NIN)); TRY(alloc(&s->diag, n));
    TRY(alloc(&s->G, n * 49)); TRY(alloc(&s->c, n * 7)); TRY(alloc(&s->d, n));
    TRY(alloc(&s->e, n)); TRY(alloc(&s->r, n)); TRY(alloc(&s->part, 4096));
    TRY(alloc(&s->master, NPARAM)); TRY(alloc(&s->bf, NPARAM)); TRY(alloc(&s->m1, NPARAM)); TRY(alloc(&s->m2, NPARAM));
    TRY(alloc(&s->out, n * NOUT)); TRY(alloc(&s->gout, n * NOUT)); TRY(alloc(&s->grad, NPARAM));
    int sms = 1, dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    s->bwd_grid = (int)std::max<long long>(1, std::min<long long>((n + BT - 1) / BT, (long long)sms));
    TRY(alloc(&s->gpart, (size_t)s->bwd_grid * NPARAM));
    TRY(check(cudaMemset(s->G, 0, n * 49 * sizeof(float))));
    TRY(check(cudaMemset(s->c, 0, n * 7 * sizeof(float))));
    TRY(check(cudaMemset(s->d, 0, n * sizeof(float))));
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
    TRY(check(cudaFuncSetAttribute(k_mlp_backward, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(BwdSmem))));
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
    return forward_and_loss(s, loss, false);
}

int cbg_spai_train(cbg_spai* s, int steps, double lr, double* loss_first, double* loss_last)
{
    if (!s || steps < 0 || !(lr > 0.0) || s->npairs < 1) return CBG_ERR_ARG;
    double l0 = 0.0, l = 0.0;
    for (int it = 0; it < steps; it++) {
        int rc = forward_and_loss(s, &l, true);
        if (rc) return rc;
        if (it == 0) l0 = l;
        k_mlp_backward<<<s->bwd_grid, BWD_THREADS, sizeof(BwdSmem), s->stream>>>(s->n, s->feat, s->bf, s->gout, s->gpart);
        k_grad_reduce<<<(NPARAM + 255) / 256, 256, 0, s->stream>>>(s->gpart, s->bwd_grid, s->grad);
        s->step++;
        k_adam<<<(NPARAM + 255) / 256, 256, 0, s->stream>>>(s->master, s->bf, s->grad, s->m1, s->m2, s->step,
                                                            (float)lr, 0.9f, 0.999f, 1e-8f);
        rc = check(cudaGetLastError());
        if (rc) return rc;
    }
    int rc = forward_and_loss(s, &l, false);
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
    k_mlp_forward<<<g, LT, 0, s->stream>>>(s->n, s->feat, s->bf, s->out);
    k_spai_pvals<<<g, LT, 0, s->stream>>>(s->rowptr, s->slot, s->n, s->out, s->diag, pvals);
    int rc = check(cudaGetLastError());
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

// ---- test access: one forward / backward with given FP32 parameters (rounded to BF16)
int cbg_mlp_forward(int64_t rows, const float* feat, const float* params_host, float* out, void* stream)
{
    if (rows < 1 || !feat || !params_host || !out) return CBG_ERR_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    float *m = nullptr, *b = nullptr;
    int rc = alloc(&m, NPARAM);
    if (!rc) rc = alloc(&b, NPARAM);
    if (!rc) rc = check(cudaMemcpyAsync(m, params_host, NPARAM * sizeof(float), cudaMemcpyHostToDevice, st));
    if (!rc) {
        k_round_bf16<<<32, 256, 0, st>>>(m, b);
        k_mlp_forward<<<grid_rows(rows), LT, 0, st>>>(rows, feat, b, out);
        rc = check(cudaGetLastError());
        if (!rc) rc = check(cudaStreamSynchronize(st));
    }
    cudaFree(m);
    cudaFree(b);
    return rc;
}

int cbg_mlp_backward(int64_t rows, const float* feat, const float* params_host, const float* gout, double* grad_host,
                     void* stream)
{
    if (rows < 1 || !feat || !params_host || !gout || !grad_host) return CBG_ERR_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    int sms = 1, dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int grid = (int)std::max<long long>(1, std::min<long long>((rows + BT - 1) / BT, sms));
    float *m = nullptr, *b = nullptr, *gp = nullptr;
    double* g = nullptr;
    int rc = alloc(&m, NPARAM);
    if (!rc) rc = alloc(&b, NPARAM);
    if (!rc) rc = alloc(&gp, (size_t)grid * NPARAM);
    if (!rc) rc = alloc(&g, NPARAM);
    if (!rc) rc = check(cudaFuncSetAttribute(k_mlp_backward, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(BwdSmem)));
    if (!rc) rc = check(cudaMemcpyAsync(m, params_host, NPARAM * sizeof(float), cudaMemcpyHostToDevice, st));
    if (!rc) {
        k_round_bf16<<<32, 256, 0, st>>>(m, b);
        k_mlp_backward<<<grid, BWD_THREADS, sizeof(BwdSmem), st>>>(rows, feat, b, gout, gp);
        k_grad_reduce<<<(NPARAM + 255) / 256, 256, 0, st>>>(gp, grid, g);
        rc = check(cudaGetLastError());
        if (!rc) rc = check(cudaMemcpyAsync(grad_host, g, NPARAM * sizeof(double), cudaMemcpyDeviceToHost, st));
        if (!rc) rc = check(cudaStreamSynchronize(st));
    }
    cudaFree(m); cudaFree(b); cudaFree(gp); cudaFree(g);
    return rc;
}

}  // extern "C"
