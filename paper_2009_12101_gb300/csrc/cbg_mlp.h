// cbg_mlp.h -- shape and parameter layout of the learned preconditioner's per-row network
// (7 stencil features -> 64 -> 64 -> 7, ReLU), shared by its host code and its kernels.
#pragma once
#include <cuda_runtime.h>

namespace cbg {

constexpr int NIN = 7, NH = 64, NOUT = 7;
// parameters, row-major (out x in): W1[64][7], b1[64], W2[64][64], b2[64], W3[7][64], b3[7]
constexpr int OFF_W1 = 0, OFF_B1 = OFF_W1 + NH * NIN, OFF_W2 = OFF_B1 + NH, OFF_B2 = OFF_W2 + NH * NH,
              OFF_W3 = OFF_B2 + NH, OFF_B3 = OFF_W3 + NOUT * NH, NPARAM = OFF_B3 + NOUT;   // 5127
constexpr int MLP_ROWS = 128;   // rows per tile of the tensor-core kernel (one per tensor-memory lane)

// What one launch of the tensor-core network kernel computes.
enum MlpMode { MLP_FWD = 0, MLP_BWD = 1, MLP_TRAIN = 2 };

struct MlpArgs {
    long long n;                  // rows
    const float* feat;            // n x 7 features (16-byte aligned)
    const float* params;          // [NPARAM] parameters, BF16 values held in FP32
    float* out;                   // MLP_FWD: n x 7 outputs
    const float* gout;            // MLP_BWD: n x 7, dL/dout (16-byte aligned)
    // MLP_TRAIN: per-row statistics of the (r, e) pairs, rows padded to a multiple of
    // MLP_ROWS (G: 49, c: 7, d, diag, mask per row; the padding rows zero)
    const float* G;
    const float* c;
    const float* d;
    const double* diag;
    const unsigned char* mask;
    double inv_npairs;
    float* gpart;                 // MLP_BWD / MLP_TRAIN: [gridDim.x][NPARAM] gradient partials
    double* lpart;                // MLP_TRAIN: [gridDim.x] loss partials
    int* fault;                   // set when a wait on the tensor core ran out (may be null)
};

// Launch the tensor-core network kernel (one CTA per SM at most, grid <= ceil(n / 128)).
cudaError_t mlp_tc_launch(int mode, int grid, cudaStream_t s, const MlpArgs& a);
int mlp_tc_grid(long long n);

}  // namespace cbg
