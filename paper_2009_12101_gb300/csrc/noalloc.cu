// noalloc.cu -- basis dot product h = V^T w that allocates no device memory.
//
// cbg_basis_dot allocates its scratch (per-block partial sums, the last-block counter,
// device copies of the scales and of the result) with cudaMalloc and frees it with
// cudaFree on every call.  Some callers cannot do that: an application whose device
// memory is owned by another allocator (a framework's caching allocator or a
// pre-sized pool) may have no memory left for a library's private cudaMalloc, and a
// latency-critical loop cannot afford cudaFree, which synchronises the whole device.
// cbg_basis_dot_noalloc takes the same arguments and keeps its scratch in one
// file-scope device array instead.  Every GPU that loads this library holds that array
// (NOALLOC_SCRATCH_BYTES, about 765 KiB) until the process exits.
#include <cuda_runtime.h>

#include <algorithm>

#include "../../include/cbgmres.h"
#include "cbg_launch.h"

using namespace cbg;

namespace {

constexpr int NOALLOC_MAX_COLS = MAXCOLS;   // columns of V per call (320)
constexpr int NOALLOC_MAX_GRID = 304;       // thread blocks of the dot kernel per call
// partial sums [grid][MAXCOLS] | scales [MAXCOLS] | result [MAXCOLS] | counter
constexpr size_t OFF_PART = 0;
constexpr size_t OFF_SCALES = (size_t)NOALLOC_MAX_GRID * MAXCOLS;
constexpr size_t OFF_OUT = OFF_SCALES + MAXCOLS;
constexpr size_t OFF_COUNTER = OFF_OUT + MAXCOLS;
constexpr size_t NOALLOC_DOUBLES = OFF_COUNTER + 32;
constexpr size_t NOALLOC_SCRATCH_BYTES = NOALLOC_DOUBLES * sizeof(double);
static_assert(NOALLOC_SCRATCH_BYTES < (1u << 20), "keep the resident scratch modest");

static __device__ __align__(256) double g_noalloc_scratch[NOALLOC_DOUBLES];

// Device address of g_noalloc_scratch on the current device, looked up on every call
// (cheap next to the call's synchronisation, and never stale: a device reset reloads the
// module and moves the array).  The host-side name g_noalloc_scratch is only a stand-in
// for the symbol and must never be handed to a kernel.
int scratch_for_current_device(double** out)
{
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return CBG_ERR_CUDA;
    *out = static_cast<double*>(p);
    return CBG_OK;
}

template <int F> int occupancy_dot() { return Launcher<F>::occupancy_dot(); }

void dot_launch(int fmt, int arith, int grid, cudaStream_t s, const DotArgs& a)
{
    switch (fmt) {
    case CBG_F64: Launcher<F64>::dot(arith, grid, s, a); break;
    case CBG_F32: Launcher<F32>::dot(arith, grid, s, a); break;
    case CBG_F16: Launcher<F16>::dot(arith, grid, s, a); break;
    case CBG_BF16: Launcher<BF16>::dot(arith, grid, s, a); break;
    case CBG_E4M3: Launcher<E4M3>::dot(arith, grid, s, a); break;
    case CBG_I32: Launcher<I32>::dot(arith, grid, s, a); break;
    default: Launcher<I16>::dot(arith, grid, s, a); break;
    }
}

int dot_occupancy(int fmt)
{
    switch (fmt) {
    case CBG_F64: return occupancy_dot<F64>();
    case CBG_F32: return occupancy_dot<F32>();
    case CBG_F16: return occupancy_dot<F16>();
    case CBG_BF16: return occupancy_dot<BF16>();
    case CBG_E4M3: return occupancy_dot<E4M3>();
    case CBG_I32: return occupancy_dot<I32>();
    default: return occupancy_dot<I16>();
    }
}

}  // namespace

extern "C" int cbg_basis_dot_noalloc(int fmt, int arith, int64_t n, int ncols, const void* V, int64_t ld,
                                     const double* scales, const double* w, double* h, void* stream)
{
    if (cbgmres_format_bytes(fmt) == 0 || (arith != CBG_ARITH_DF32 && arith != CBG_ARITH_FP64) || n < 1 ||
        ncols < 1 || !V || ld < n || ld % TILE_ROWS || !scales || !w || !h)
        return CBG_ERR_ARG;
    if (ncols > NOALLOC_MAX_COLS) return CBG_ERR_ARG;   // beyond the static scratch
    double* base = nullptr;
    int rc = scratch_for_current_device(&base);
    if (rc) return rc;
    int dev = 0, sms = 1;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return CBG_ERR_CUDA;
    const long long tiles = ld / DOT_MIN_ROWS;
    const int grid = (int)std::max<long long>(
        1, std::min<long long>({tiles, (long long)sms * std::max(1, dot_occupancy(fmt)), (long long)NOALLOC_MAX_GRID}));
    cudaStream_t s = (cudaStream_t)stream;
    double* part = base + OFF_PART;
    double* sc = base + OFF_SCALES;
    double* out = base + OFF_OUT;
    unsigned int* counter = reinterpret_cast<unsigned int*>(base + OFF_COUNTER);
    // the last-block counter must start at zero; the other regions are overwritten
    if (cudaMemsetAsync(counter, 0, sizeof(unsigned int), s) != cudaSuccess ||
        cudaMemcpyAsync(sc, scales, ncols * sizeof(double), cudaMemcpyHostToDevice, s) != cudaSuccess)
        return CBG_ERR_CUDA;
    DotArgs a{};
    a.V = static_cast<const unsigned char*>(V);
    a.ldb = ld * cbgmres_format_bytes(fmt);
    a.ncols = ncols;
    a.scales = sc;
    a.w = w;
    a.nrows = ld;
    a.part = part;
    a.counter = counter;
    a.out = out;
    dot_launch(fmt, arith, grid, s, a);
    if (cudaGetLastError() != cudaSuccess ||
        cudaMemcpyAsync(h, out, ncols * sizeof(double), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return CBG_ERR_CUDA;
    return CBG_OK;
}
