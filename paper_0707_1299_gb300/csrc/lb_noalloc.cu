// lb_noalloc.cu -- lb_totals_noalloc: the FP64 totals reduction of the
// moments kernel for callers that cannot allocate device memory.
//
// Who needs it: code whose device memory is owned entirely by its own pool
// allocator (a framework's caching allocator, a fixed arena sized up front)
// and must not go around it, and code that cannot afford cudaMalloc /
// cudaFree at all -- cudaFree waits for the whole device, which stalls any
// other work the caller keeps in flight, and an allocation can fail with
// out-of-memory in the middle of a long run.  Such a caller cannot create an
// lb_ctx (lb_create allocates), but it can hold a population array of its
// own and still ask for the conserved totals of it.
//
// Scratch: the per-block partial sums live in the file-scope array below,
// which every GPU that loads this library keeps until the process exits.
// Host code cannot use the array's name as a device address; the address
// is looked up with cudaGetSymbolAddress (with the device current).  Every
// call that is not being captured into a CUDA graph looks it up again, so a
// device reset or a new primary context (which may load the module at
// another address) never leaves a stale pointer behind; a call made while
// its stream is capturing takes the address the last uncaptured call on
// that device found, so the first call on a device must come before any
// stream capture there.
// All calls share the array and it keeps the previous call's contents: each
// block overwrites its own slot before the final reduction reads it, so
// nothing needs clearing, but two calls whose work overlaps on the GPU
// (different streams, or different host threads on the same device) race on
// it and may return wrong totals.
#include <math.h>

#include <mutex>

#include "../../include/lb.h"
#include "lb_internal.h"

namespace {

constexpr int NA_WARPS = 4;
constexpr int NA_MAX_BLOCKS = 1024;  // partial sums held in the static array
constexpr int NA_MAX_DEVICES = 64;

static __device__ __align__(256) double g_totals_scratch[4 * NA_MAX_BLOCKS];

std::mutex g_setup_mutex;
double* g_scratch_ptr[NA_MAX_DEVICES] = {nullptr};

__device__ __forceinline__ double na_block_sum(double v, double* sh) {
    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    __syncthreads();
    if (lane == 0) sh[w] = v;
    __syncthreads();
    double t = 0.0;
    if (threadIdx.x == 0)
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) t += sh[i];
    return t;  // valid in thread 0
}

// Each warp takes 32-site x-row tiles in a grid-stride loop; every block
// writes its four partial sums (rho, rho u) to its slot of `partials`.
template <typename S, bool WALLS>
__global__ void __launch_bounds__(NA_WARPS * 32)
k_totals_partials(const lbk::Pops<S> src, lbk::Geom g, lbk::UForce<typename lbk::Store<S>::T> fu, float inv_scale,
                  double* __restrict__ partials) {
    using T = typename lbk::Store<S>::T;
    __shared__ double sh[NA_WARPS];
    const int lane = threadIdx.x & 31;
    double acc[4] = {0.0, 0.0, 0.0, 0.0};
    for (long long tile = (long long)blockIdx.x * NA_WARPS + (threadIdx.x >> 5); tile < g.ntiles;
         tile += (long long)gridDim.x * NA_WARPS) {
        const int tx = (int)(tile % g.ntx);
        const long long r = tile / g.ntx;
        const int y = (int)(r % g.ny), z = (int)(r / g.ny);
        const int x = tx * lbk::TILE_X + lane;
        if (x >= g.nx || (WALLS && lbk::is_solid(g, z))) continue;
        const lbk::Nbr nb = lbk::neighbours(g, x, y, z);
        T f[lbk::NQ];
        lbk::pull19<S, WALLS>(src, nb, f);
        lbk::unscale19<S>(f, inv_scale);
        T drho, vx, vy, vz;
        lbk::macro19<T, lbk::Store<S>::kCompensate>(f, fu.F[0], fu.F[1], fu.F[2], drho, vx, vy, vz);
        const double rho = 1.0 + (double)drho;
        acc[0] += rho;
        acc[1] += rho * (double)vx;
        acc[2] += rho * (double)vy;
        acc[3] += rho * (double)vz;
    }
    for (int a = 0; a < 4; ++a) {
        const double t = na_block_sum(acc[a], sh);
        if (threadIdx.x == 0) partials[4 * blockIdx.x + a] = t;
    }
}

__global__ void k_totals_final(const double* __restrict__ partials, int nblocks, double* __restrict__ out) {
    __shared__ double sh[32];
    for (int a = 0; a < 4; ++a) {
        double v = 0.0;
        for (int b = threadIdx.x; b < nblocks; b += blockDim.x) v += partials[4 * b + a];
        const double t = na_block_sum(v, sh);
        if (threadIdx.x == 0) out[a] = t;
    }
}

template <typename S>
cudaError_t launch_totals(const void* df, const lbk::Geom& g, const double F[3], float inv_scale, double* scratch,
                          double* totals, cudaStream_t stream) {
    using T = typename lbk::Store<S>::T;
    lbk::Pops<S> src;
    for (int i = 0; i < lbk::NQ; ++i) src.p[i] = (S*)df + (size_t)i * (size_t)g.V;
    lbk::UForce<T> fu;
    for (int a = 0; a < 3; ++a) fu.F[a] = (T)F[a];
    const long long want = (g.ntiles + NA_WARPS - 1) / NA_WARPS;
    const int blocks = (int)(want < NA_MAX_BLOCKS ? want : NA_MAX_BLOCKS);
    const bool walls = g.wall_lo >= 0 || g.wall_hi >= 0;
    if (walls)
        k_totals_partials<S, true><<<blocks, NA_WARPS * 32, 0, stream>>>(src, g, fu, inv_scale, scratch);
    else
        k_totals_partials<S, false><<<blocks, NA_WARPS * 32, 0, stream>>>(src, g, fu, inv_scale, scratch);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_totals_final<<<1, 256, 0, stream>>>(scratch, blocks, totals);
    return cudaGetLastError();
}

}  // namespace

extern "C" lb_status lb_totals_noalloc(const void* df, int precision, const int grid[3], int z_lo, int z_hi,
                                       const double F[3], double* totals, void* stream) {
    if (!df || !grid || !totals) return LB_ERR_ARG;
    if (precision < LB_F64 || precision > LB_BF16S) return LB_ERR_ARG;
    for (int a = 0; a < 3; ++a)
        if (grid[a] < 1) return LB_ERR_ARG;
    const long long V = (long long)grid[0] * grid[1] * grid[2];
    if (V >= (1LL << 32)) return LB_ERR_ARG;  // beyond the 32-bit site indexing of the kernels
    if (z_lo < -1 || z_lo >= grid[2] || z_hi < -1 || z_hi >= grid[2]) return LB_ERR_ARG;
    double Fu[3] = {0.0, 0.0, 0.0};
    if (F)
        for (int a = 0; a < 3; ++a) {
            if (!isfinite(F[a])) return LB_ERR_NONFINITE;
            Fu[a] = F[a];
        }

    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= NA_MAX_DEVICES) return LB_ERR_CUDA;
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing((cudaStream_t)stream, &cap) != cudaSuccess) {
        cudaGetLastError();
        return LB_ERR_CUDA;
    }
    double* scratch = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_setup_mutex);
        if (cap == cudaStreamCaptureStatusNone) {  // refresh: the module may have moved since the last call
            void* p = nullptr;
            if (cudaGetSymbolAddress(&p, g_totals_scratch) != cudaSuccess || !p) {
                cudaGetLastError();
                return LB_ERR_CUDA;
            }
            g_scratch_ptr[dev] = (double*)p;
        }
        scratch = g_scratch_ptr[dev];
    }
    if (!scratch) return LB_ERR_STATE;  // captured before any uncaptured call on this device

    lbk::Geom g;
    g.nx = grid[0];
    g.ny = grid[1];
    g.nz = grid[2];
    g.ntx = (grid[0] + lbk::TILE_X - 1) / lbk::TILE_X;
    g.plane = (unsigned)grid[0] * (unsigned)grid[1];
    g.V = V;
    g.ntiles = (long long)g.ntx * grid[1] * grid[2];
    g.wall_lo = z_lo;
    g.wall_hi = z_hi;
    const float inv_scale = precision == LB_F16S ? 1.0f / 1048576.0f : 1.0f;
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e;
    switch (precision) {
        case LB_F64: e = launch_totals<double>(df, g, Fu, inv_scale, scratch, totals, s); break;
        case LB_F32: e = launch_totals<float>(df, g, Fu, inv_scale, scratch, totals, s); break;
        case LB_F16S: e = launch_totals<__half>(df, g, Fu, inv_scale, scratch, totals, s); break;
        default: e = launch_totals<__nv_bfloat16>(df, g, Fu, inv_scale, scratch, totals, s); break;
    }
    return e == cudaSuccess ? LB_OK : LB_ERR_CUDA;
}
