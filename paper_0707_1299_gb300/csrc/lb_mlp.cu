// lb_mlp.cu -- the learned correction of the interpolated colloid velocity:
// neighbour features (cell list), and a 27 -> 64 -> 64 -> 3 SiLU perceptron
// in bfloat16 with FP32 accumulation (forward, fused forward + backward,
// Adam), all hand-written.
//
// Rounding points (the training oracle mirrors them): the input x, the
// weight matrices and the activations h1, h2 are rounded to bfloat16 (round
// to nearest even) before they enter a product; pre-activations, biases,
// accumulations and gradients are FP32; master weights and Adam moments are
// FP32.
#include <math.h>
#include <stdint.h>

#include <new>
#include <string>

#include "../../include/lb.h"
#include "lb_internal.h"

namespace {

using lbk::Geom;

constexpr int D0 = 27, D1 = 64, D2 = 64, D3 = 3;
constexpr int OFF_W1 = 0, OFF_B1 = OFF_W1 + D1 * D0, OFF_W2 = OFF_B1 + D1, OFF_B2 = OFF_W2 + D2 * D1,
              OFF_W3 = OFF_B2 + D2, OFF_B3 = OFF_W3 + D3 * D2, NPARAM = OFF_B3 + D3;
constexpr int TS = 64;        // samples per tile
constexpr int NT = 256;       // threads per block
constexpr int P2 = 65;        // padded row length of 64-wide smem arrays
constexpr float FEAT_LENGTH = 4.0f;
constexpr float R_CUT = 8.0f;
constexpr int NNB = 8;

__device__ __forceinline__ float bf16r(float v) { return __bfloat162float(__float2bfloat16_rn(v)); }
__device__ __forceinline__ float silu(float z) { return z / (1.0f + expf(-z)); }
__device__ __forceinline__ float dsilu(float z) {
    const float s = 1.0f / (1.0f + expf(-z));
    return s * (1.0f + z * (1.0f - s));
}

// shared-memory layout (floats)
struct Smem {
    static constexpr int W1 = 0;                    // [64][27]
    static constexpr int W2 = W1 + D1 * D0;         // [64][65]
    static constexpr int W3 = W2 + D2 * P2;         // [3][64]
    static constexpr int B = W3 + D3 * D2;          // b1 b2 b3
    static constexpr int X = B + D1 + D2 + D3;      // [64][28]
    static constexpr int Z1 = X + TS * 28;          // [64][65]
    static constexpr int H1 = Z1 + TS * P2;
    static constexpr int Z2 = H1 + TS * P2;
    static constexpr int H2 = Z2 + TS * P2;
    static constexpr int GY = H2 + TS * P2;         // [64][3]
    static constexpr int GZ2 = GY + TS * D3;        // [64][65]
    static constexpr int GZ1 = GZ2 + TS * P2;       // [64][65]
    static constexpr int END = GZ1 + TS * P2;
    static constexpr int FWD_END = GY + TS * D3;    // forward-only kernels stop here (tile_forward stages y in GY)
};

__device__ void load_weights(const float* __restrict__ p, float* sm) {
    for (int i = threadIdx.x; i < D1 * D0; i += NT) sm[Smem::W1 + i] = bf16r(p[OFF_W1 + i]);
    for (int i = threadIdx.x; i < D2 * D1; i += NT) sm[Smem::W2 + (i / D1) * P2 + i % D1] = bf16r(p[OFF_W2 + i]);
    for (int i = threadIdx.x; i < D3 * D2; i += NT) sm[Smem::W3 + i] = bf16r(p[OFF_W3 + i]);
    for (int i = threadIdx.x; i < D1; i += NT) sm[Smem::B + i] = p[OFF_B1 + i];
    for (int i = threadIdx.x; i < D2; i += NT) sm[Smem::B + D1 + i] = p[OFF_B2 + i];
    for (int i = threadIdx.x; i < D3; i += NT) sm[Smem::B + D1 + D2 + i] = p[OFF_B3 + i];
}

// Forward pass of one tile of `ns` samples (rows >= ns are zero and unused).
__device__ void tile_forward(const float* __restrict__ feat, long long s0, int ns, float* sm, float* __restrict__ y_out) {
    for (int i = threadIdx.x; i < TS * 28; i += NT) {
        const int s = i / 28, k = i % 28;
        sm[Smem::X + i] = (s < ns && k < D0) ? bf16r(feat[(s0 + s) * D0 + k]) : 0.0f;
    }
    __syncthreads();
    const int j = threadIdx.x & 63, sg = threadIdx.x >> 6;  // unit j, sample group sg (16 samples each)
    for (int m = 0; m < TS / 4; ++m) {
        const int s = sg + 4 * m;
        float z = sm[Smem::B + j];
        for (int k = 0; k < D0; ++k) z = fmaf(sm[Smem::X + s * 28 + k], sm[Smem::W1 + j * D0 + k], z);
        sm[Smem::Z1 + s * P2 + j] = z;
        sm[Smem::H1 + s * P2 + j] = bf16r(silu(z));
    }
    __syncthreads();
    for (int m = 0; m < TS / 4; ++m) {
        const int s = sg + 4 * m;
        float z = sm[Smem::B + D1 + j];
        for (int k = 0; k < D1; ++k) z = fmaf(sm[Smem::H1 + s * P2 + k], sm[Smem::W2 + j * P2 + k], z);
        sm[Smem::Z2 + s * P2 + j] = z;
        sm[Smem::H2 + s * P2 + j] = bf16r(silu(z));
    }
    __syncthreads();
    if (threadIdx.x < TS * D3) {
        const int s = threadIdx.x / D3, o = threadIdx.x % D3;
        float yv = sm[Smem::B + D1 + D2 + o];
        for (int k = 0; k < D2; ++k) yv = fmaf(sm[Smem::H2 + s * P2 + k], sm[Smem::W3 + o * D2 + k], yv);
        if (y_out && s < ns) y_out[(s0 + s) * D3 + o] = yv;
        sm[Smem::GY + threadIdx.x] = yv;  // the backward pass turns it into dL/dy
    }
    __syncthreads();
}

__global__ void __launch_bounds__(NT) km_forward(const float* __restrict__ params, long long n,
                                                 const float* __restrict__ feat, float* __restrict__ out) {
    extern __shared__ float sm[];
    load_weights(params, sm);
    __syncthreads();
    for (long long t = blockIdx.x; t * TS < n; t += gridDim.x) {
        const long long s0 = t * TS;
        const int ns = (int)(n - s0 < TS ? n - s0 : TS);
        tile_forward(feat, s0, ns, sm, out);
    }
}

// Forward + backward of the mean squared error (1 / 3n) sum (y - t)^2 over
// all n samples; gradients and the sum of squared errors are accumulated
// into grad[NPARAM] and sse[0] (both cleared by the caller).
__global__ void __launch_bounds__(NT) km_grad(const float* __restrict__ params, long long n,
                                              const float* __restrict__ feat, const float* __restrict__ target,
                                              float* __restrict__ grad, float* __restrict__ sse) {
    extern __shared__ float sm[];
    load_weights(params, sm);
    __syncthreads();
    const float gscale = 2.0f / (3.0f * (float)n);
    // per-thread accumulators of the weight gradients it owns
    float aW2[16], aW1[7], aW3 = 0.f, ab2 = 0.f, ab1 = 0.f, ab3 = 0.f, asse = 0.f;
    for (int q = 0; q < 16; ++q) aW2[q] = 0.f;
    for (int q = 0; q < 7; ++q) aW1[q] = 0.f;
    const int j = threadIdx.x & 63, sg = threadIdx.x >> 6;
    for (long long t = blockIdx.x; t * TS < n; t += gridDim.x) {
        const long long s0 = t * TS;
        const int ns = (int)(n - s0 < TS ? n - s0 : TS);
        tile_forward(feat, s0, ns, sm, nullptr);
        if (threadIdx.x < TS * D3) {  // dL/dy
            const int s = threadIdx.x / D3, o = threadIdx.x % D3;
            float g = 0.f;
            if (s < ns) {
                const float d = sm[Smem::GY + threadIdx.x] - target[(s0 + s) * D3 + o];
                asse = fmaf(d, d, asse);
                g = gscale * d;
            }
            sm[Smem::GY + threadIdx.x] = g;
        }
        __syncthreads();
        // layer 3: gW3[o][k] = sum_s gy[s][o] h2[s][k]; gb3
        if (threadIdx.x < D3 * D2) {
            const int o = threadIdx.x / D2, k = threadIdx.x % D2;
            float a = 0.f;
            for (int s = 0; s < TS; ++s) a = fmaf(sm[Smem::GY + s * D3 + o], sm[Smem::H2 + s * P2 + k], a);
            aW3 += a;
        }
        if (threadIdx.x < D3) {
            float a = 0.f;
            for (int s = 0; s < TS; ++s) a += sm[Smem::GY + s * D3 + threadIdx.x];
            ab3 += a;
        }
        // gz2[s][j] = (sum_o gy[s][o] W3[o][j]) dsilu(z2[s][j])
        for (int m = 0; m < TS / 4; ++m) {
            const int s = sg + 4 * m;
            float g = 0.f;
            for (int o = 0; o < D3; ++o) g = fmaf(sm[Smem::GY + s * D3 + o], sm[Smem::W3 + o * D2 + j], g);
            sm[Smem::GZ2 + s * P2 + j] = g * dsilu(sm[Smem::Z2 + s * P2 + j]);
        }
        __syncthreads();
        // layer 2: gW2[j][k] = sum_s gz2[s][j] h1[s][k]; thread owns k = j (its unit) for 16 rows
        for (int q = 0; q < 16; ++q) {
            const int row = sg + 4 * q;  // output unit
            float a = 0.f;
            for (int s = 0; s < TS; ++s) a = fmaf(sm[Smem::GZ2 + s * P2 + row], sm[Smem::H1 + s * P2 + j], a);
            aW2[q] += a;
        }
        if (threadIdx.x < D2) {
            float a = 0.f;
            for (int s = 0; s < TS; ++s) a += sm[Smem::GZ2 + s * P2 + threadIdx.x];
            ab2 += a;
        }
        // gz1[s][j] = (sum_i gz2[s][i] W2[i][j]) dsilu(z1[s][j])
        for (int m = 0; m < TS / 4; ++m) {
            const int s = sg + 4 * m;
            float g = 0.f;
            for (int i = 0; i < D2; ++i) g = fmaf(sm[Smem::GZ2 + s * P2 + i], sm[Smem::W2 + i * P2 + j], g);
            sm[Smem::GZ1 + s * P2 + j] = g * dsilu(sm[Smem::Z1 + s * P2 + j]);
        }
        __syncthreads();
        // layer 1: gW1[u][k] = sum_s gz1[s][u] x[s][k]; entries e = threadIdx.x + 256 q
        for (int q = 0; q < 7; ++q) {
            const int e = threadIdx.x + NT * q;
            if (e < D1 * D0) {
                const int u = e / D0, k = e % D0;
                float a = 0.f;
                for (int s = 0; s < TS; ++s) a = fmaf(sm[Smem::GZ1 + s * P2 + u], sm[Smem::X + s * 28 + k], a);
                aW1[q] += a;
            }
        }
        if (threadIdx.x < D1) {
            float a = 0.f;
            for (int s = 0; s < TS; ++s) a += sm[Smem::GZ1 + s * P2 + threadIdx.x];
            ab1 += a;
        }
        __syncthreads();
    }
    for (int q = 0; q < 16; ++q) atomicAdd(&grad[OFF_W2 + (sg + 4 * q) * D1 + j], aW2[q]);
    for (int q = 0; q < 7; ++q) {
        const int e = threadIdx.x + NT * q;
        if (e < D1 * D0) atomicAdd(&grad[OFF_W1 + e], aW1[q]);
    }
    if (threadIdx.x < D3 * D2) atomicAdd(&grad[OFF_W3 + threadIdx.x], aW3);
    if (threadIdx.x < D3) atomicAdd(&grad[OFF_B3 + threadIdx.x], ab3);
    if (threadIdx.x < D2) atomicAdd(&grad[OFF_B2 + threadIdx.x], ab2);
    if (threadIdx.x < D1) atomicAdd(&grad[OFF_B1 + threadIdx.x], ab1);
    for (int off = 16; off > 0; off >>= 1) asse += __shfl_xor_sync(0xffffffffu, asse, off);
    if ((threadIdx.x & 31) == 0) atomicAdd(sse, asse);
}

__global__ void km_adam(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m,
                        float* __restrict__ v, float lr, float b1, float b2, float eps, float c1, float c2) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= NPARAM) return;
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

// --------------------------------------------------------- features
__device__ __forceinline__ int cell_of(double X, double box, int nc) {
    int c = (int)(X / box * nc);
    return c < 0 ? 0 : (c >= nc ? nc - 1 : c);
}

__global__ void kf_count(const double* __restrict__ pos, long long n, Geom g, int3 nc, int* __restrict__ count,
                         int* __restrict__ cell) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int cx = cell_of(pos[3 * i], g.nx, nc.x), cy = cell_of(pos[3 * i + 1], g.ny, nc.y),
              cz = cell_of(pos[3 * i + 2], g.nz, nc.z);
    const int c = (cz * nc.y + cy) * nc.x + cx;
    cell[i] = c;
    atomicAdd(&count[c], 1);
}

// exclusive scan of count[0..m) into start[0..m], one block
__global__ void kf_scan(const int* __restrict__ count, int m, int* __restrict__ start) {
    __shared__ int part[1024];
    const int per = (m + blockDim.x - 1) / blockDim.x;
    const int b = threadIdx.x * per;
    int s = 0;
    for (int i = b; i < b + per && i < m; ++i) s += count[i];
    part[threadIdx.x] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        int acc = 0;
        for (int i = 0; i < (int)blockDim.x; ++i) {
            const int t = part[i];
            part[i] = acc;
            acc += t;
        }
        start[m] = acc;
    }
    __syncthreads();
    int acc = part[threadIdx.x];
    for (int i = b; i < b + per && i < m; ++i) {
        start[i] = acc;
        acc += count[i];
    }
}

__global__ void kf_fill(long long n, const int* __restrict__ cell, const int* __restrict__ start,
                        int* __restrict__ cursor, int* __restrict__ sorted) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int c = cell[i];
    sorted[start[c] + atomicAdd(&cursor[c], 1)] = (int)i;
}

// 27 features per colloid: fractional offset, then the 8 nearest others
// within R_CUT (minimum image), nearest first, equal distances by index.
__global__ void kf_knn(const double* __restrict__ pos, long long n, Geom g, int3 nc, const int* __restrict__ start,
                       const int* __restrict__ sorted, float* __restrict__ feat) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double box[3] = {(double)g.nx, (double)g.ny, (double)g.nz};
    const double P[3] = {pos[3 * i], pos[3 * i + 1], pos[3 * i + 2]};
    double bd[NNB];
    int bj[NNB];
    float bv[NNB][3];
    for (int q = 0; q < NNB; ++q) {
        bd[q] = 1.0e300;
        bj[q] = 0x7fffffff;
    }
    const int c0[3] = {cell_of(P[0], box[0], nc.x), cell_of(P[1], box[1], nc.y), cell_of(P[2], box[2], nc.z)};
    const int ncs[3] = {nc.x, nc.y, nc.z};
    int lo[3], hi[3];
    for (int a = 0; a < 3; ++a) {  // neighbouring cells, each visited once
        if (ncs[a] >= 3) {
            lo[a] = -1;
            hi[a] = 1;
        } else {
            lo[a] = 0;
            hi[a] = ncs[a] - 1;
        }
    }
    const double rc2 = (double)R_CUT * (double)R_CUT;
    for (int dz = lo[2]; dz <= hi[2]; ++dz)
        for (int dy = lo[1]; dy <= hi[1]; ++dy)
            for (int dx = lo[0]; dx <= hi[0]; ++dx) {
                const int cx = (c0[0] + dx + ncs[0]) % ncs[0], cy = (c0[1] + dy + ncs[1]) % ncs[1],
                          cz = (c0[2] + dz + ncs[2]) % ncs[2];
                const int c = (cz * ncs[1] + cy) * ncs[0] + cx;
                for (int q = start[c]; q < start[c + 1]; ++q) {
                    const int jn = sorted[q];
                    if (jn == i) continue;
                    double d[3];
                    for (int a = 0; a < 3; ++a) {
                        d[a] = pos[3 * (long long)jn + a] - P[a];
                        d[a] -= box[a] * rint(d[a] / box[a]);
                    }
                    const double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
                    if (r2 > rc2) continue;
                    if (r2 > bd[NNB - 1] || (r2 == bd[NNB - 1] && jn > bj[NNB - 1])) continue;
                    int p = NNB - 1;  // insertion into the sorted list
                    while (p > 0 && (r2 < bd[p - 1] || (r2 == bd[p - 1] && jn < bj[p - 1]))) {
                        bd[p] = bd[p - 1];
                        bj[p] = bj[p - 1];
                        for (int a = 0; a < 3; ++a) bv[p][a] = bv[p - 1][a];
                        --p;
                    }
                    bd[p] = r2;
                    bj[p] = jn;
                    for (int a = 0; a < 3; ++a) bv[p][a] = (float)(d[a] / (double)FEAT_LENGTH);
                }
            }
    float* f = feat + i * D0;
    for (int a = 0; a < 3; ++a) f[a] = (float)(P[a] - floor(P[a]));
    for (int q = 0; q < NNB; ++q)
        for (int a = 0; a < 3; ++a) f[3 + 3 * q + a] = bd[q] < 1.0e299 ? bv[q][a] : 0.0f;
}

}  // namespace

struct lb_mlp {
    cudaStream_t stream;
    float *p, *g, *m, *v, *sse;
    long long t;              // Adam steps taken
    int *ws;                  // feature workspace (cell lists), grown on demand
    size_t ws_ints;
    int smem_fwd, smem_grad, blocks;
    std::string err;
};

namespace {

lb_status mfail(lb_mlp* net, lb_status s, const std::string& m) {
    if (net) net->err = m;
    return s;
}

#define LB_MCUDA(call, where)                                                                     \
    do {                                                                                          \
        cudaError_t e_ = (call);                                                                  \
        if (e_ != cudaSuccess)                                                                    \
            return mfail(net, e_ == cudaErrorMemoryAllocation ? LB_ERR_OOM : LB_ERR_CUDA,         \
                         std::string(where) + ": " + cudaGetErrorString(e_));                     \
    } while (0)

int grid_for(long long n) {
    const long long tiles = (n + TS - 1) / TS;
    return (int)(tiles < 152LL * 2 ? (tiles > 0 ? tiles : 1) : 152LL * 2);
}

}  // namespace

namespace lbk {

size_t mlp_features_ws_ints(long long n, const int box[3]) {
    long long m = 1;
    for (int a = 0; a < 3; ++a) m *= (box[a] / (int)R_CUT > 0 ? box[a] / (int)R_CUT : 1);
    return (size_t)(m + (m + 1) + m + 2 * n);  // count, start, cursor, cell, sorted
}

cudaError_t mlp_features(long long n, const double* pos, const int box[3], float* feat, int* ws, cudaStream_t st) {
    int3 nc;
    nc.x = box[0] / (int)R_CUT > 0 ? box[0] / (int)R_CUT : 1;
    nc.y = box[1] / (int)R_CUT > 0 ? box[1] / (int)R_CUT : 1;
    nc.z = box[2] / (int)R_CUT > 0 ? box[2] / (int)R_CUT : 1;
    const long long m = (long long)nc.x * nc.y * nc.z;
    int* count = ws;
    int* start = count + m;
    int* cursor = start + m + 1;
    int* cell = cursor + m;
    int* sorted = cell + n;
    Geom g{};
    g.nx = box[0];
    g.ny = box[1];
    g.nz = box[2];
    cudaError_t e = cudaMemsetAsync(count, 0, sizeof(int) * m, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(cursor, 0, sizeof(int) * m, st);
    if (e != cudaSuccess) return e;
    const unsigned blocks = (unsigned)((n + 255) / 256);
    kf_count<<<blocks, 256, 0, st>>>(pos, n, g, nc, count, cell);
    kf_scan<<<1, 1024, 0, st>>>(count, (int)m, start);
    kf_fill<<<blocks, 256, 0, st>>>(n, cell, start, cursor, sorted);
    kf_knn<<<blocks, 256, 0, st>>>(pos, n, g, nc, start, sorted, feat);
    return cudaGetLastError();
}

cudaError_t mlp_forward(const lb_mlp* net, long long n, const float* feat, float* out, cudaStream_t st) {
    km_forward<<<grid_for(n), NT, net->smem_fwd, st>>>(net->p, n, feat, out);
    return cudaGetLastError();
}

}  // namespace lbk

extern "C" {

int lb_mlp_num_params(void) { return NPARAM; }

lb_status lb_mlp_create(lb_mlp** out, const float* init, void* stream) {
    if (!out || !init) return LB_ERR_ARG;
    *out = nullptr;
    lb_mlp* net = new (std::nothrow) lb_mlp();
    if (!net) return LB_ERR_OOM;
    net->stream = (cudaStream_t)stream;
    net->smem_fwd = Smem::FWD_END * (int)sizeof(float);
    net->smem_grad = Smem::END * (int)sizeof(float);
    cudaError_t e = cudaMalloc(&net->p, sizeof(float) * (4 * NPARAM + 1));
    if (e == cudaSuccess) {
        net->g = net->p + NPARAM;
        net->m = net->g + NPARAM;
        net->v = net->m + NPARAM;
        net->sse = net->v + NPARAM;
        e = cudaMemsetAsync(net->p, 0, sizeof(float) * (4 * NPARAM + 1), net->stream);
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(net->p, init, sizeof(float) * NPARAM, cudaMemcpyDefault, net->stream);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(km_grad, cudaFuncAttributeMaxDynamicSharedMemorySize, net->smem_grad);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(km_forward, cudaFuncAttributeMaxDynamicSharedMemorySize, net->smem_fwd);
    if (e == cudaSuccess) e = cudaStreamSynchronize(net->stream);
    if (e != cudaSuccess) {
        lb_mlp_destroy(net);
        return e == cudaErrorMemoryAllocation ? LB_ERR_OOM : LB_ERR_CUDA;
    }
    *out = net;
    return LB_OK;
}

void lb_mlp_destroy(lb_mlp* net) {
    if (!net) return;
    cudaStreamSynchronize(net->stream);
    cudaFree(net->p);
    cudaFree(net->ws);
    delete net;
}

const char* lb_mlp_last_error(const lb_mlp* net) { return net ? net->err.c_str() : ""; }

lb_status lb_mlp_get_params(lb_mlp* net, float* out) {
    if (!net || !out) return LB_ERR_ARG;
    LB_MCUDA(cudaMemcpyAsync(out, net->p, sizeof(float) * NPARAM, cudaMemcpyDefault, net->stream), "params copy");
    LB_MCUDA(cudaStreamSynchronize(net->stream), "stream synchronize");
    return LB_OK;
}

lb_status lb_mlp_set_params(lb_mlp* net, const float* in) {
    if (!net || !in) return LB_ERR_ARG;
    LB_MCUDA(cudaMemcpyAsync(net->p, in, sizeof(float) * NPARAM, cudaMemcpyDefault, net->stream), "params copy");
    LB_MCUDA(cudaMemsetAsync(net->m, 0, sizeof(float) * 2 * NPARAM, net->stream), "adam reset");
    net->t = 0;
    LB_MCUDA(cudaStreamSynchronize(net->stream), "stream synchronize");
    return LB_OK;
}

lb_status lb_mlp_features(lb_mlp* net, long long n, const double* pos, const int box[3], float* feat) {
    if (!net || n < 0 || (n && (!pos || !feat)) || !box) return mfail(net, LB_ERR_ARG, "lb_mlp_features: bad argument");
    if (box[0] < 1 || box[1] < 1 || box[2] < 1) return mfail(net, LB_ERR_ARG, "lb_mlp_features: bad box");
    if (n == 0) return LB_OK;
    const size_t need = lbk::mlp_features_ws_ints(n, box);
    if (need > net->ws_ints) {
        cudaFree(net->ws);
        net->ws = nullptr;
        net->ws_ints = 0;
        LB_MCUDA(cudaMalloc(&net->ws, sizeof(int) * need), "feature workspace");
        net->ws_ints = need;
    }
    LB_MCUDA(lbk::mlp_features(n, pos, box, feat, net->ws, net->stream), "feature kernels");
    return LB_OK;
}

lb_status lb_mlp_forward(lb_mlp* net, long long n, const float* feat, float* out) {
    if (!net || n < 0 || (n && (!feat || !out))) return mfail(net, LB_ERR_ARG, "lb_mlp_forward: bad argument");
    if (n == 0) return LB_OK;
    LB_MCUDA(lbk::mlp_forward(net, n, feat, out, net->stream), "forward kernel");
    return LB_OK;
}

static lb_status run_grad(lb_mlp* net, long long n, const float* feat, const float* target) {
    LB_MCUDA(cudaMemsetAsync(net->g, 0, sizeof(float) * NPARAM, net->stream), "memset");
    LB_MCUDA(cudaMemsetAsync(net->sse, 0, sizeof(float), net->stream), "memset");
    km_grad<<<grid_for(n), NT, net->smem_grad, net->stream>>>(net->p, n, feat, target, net->g, net->sse);
    LB_MCUDA(cudaGetLastError(), "gradient kernel");
    return LB_OK;
}

lb_status lb_mlp_grad(lb_mlp* net, long long n, const float* feat, const float* target, float* grad, float* sse) {
    if (!net || n < 1 || !feat || !target) return mfail(net, LB_ERR_ARG, "lb_mlp_grad: bad argument");
    lb_status s = run_grad(net, n, feat, target);
    if (s != LB_OK) return s;
    if (grad) LB_MCUDA(cudaMemcpyAsync(grad, net->g, sizeof(float) * NPARAM, cudaMemcpyDefault, net->stream), "copy");
    if (sse) LB_MCUDA(cudaMemcpyAsync(sse, net->sse, sizeof(float), cudaMemcpyDefault, net->stream), "copy");
    LB_MCUDA(cudaStreamSynchronize(net->stream), "stream synchronize");
    return LB_OK;
}

lb_status lb_mlp_train_step(lb_mlp* net, long long n, const float* feat, const float* target, float lr, float* sse) {
    if (!net || n < 1 || !feat || !target || !(lr > 0)) return mfail(net, LB_ERR_ARG, "lb_mlp_train_step: bad argument");
    lb_status s = run_grad(net, n, feat, target);
    if (s != LB_OK) return s;
    net->t += 1;
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = 1.0f - powf(b1, (float)net->t), c2 = 1.0f - powf(b2, (float)net->t);
    km_adam<<<(NPARAM + 255) / 256, 256, 0, net->stream>>>(net->p, net->g, net->m, net->v, lr, b1, b2, 1e-8f, c1, c2);
    LB_MCUDA(cudaGetLastError(), "adam kernel");
    if (sse) LB_MCUDA(cudaMemcpyAsync(sse, net->sse, sizeof(float), cudaMemcpyDefault, net->stream), "copy");
    return LB_OK;
}

}  // extern "C"
