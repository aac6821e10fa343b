// lb_mlp.cu -- the learned correction of the interpolated colloid velocity:
// neighbour features (cell list), and a 27 -> 64 -> 64 -> 3 SiLU perceptron
// in bfloat16 with FP32 accumulation on the tensor cores (forward, fused
// forward + backward), Adam, all hand-written.
//
// Rounding points (the training oracle mirrors them): every operand of a
// product is bfloat16 (round to nearest even) -- the input x, the weight
// matrices, the activations h1, h2, and in the backward pass dL/dy and the
// pre-activation gradients gz2, gz1 where they enter the weight-gradient and
// gh1 products; gh2 = (dL/dy) W3 takes the FP32 dL/dy.  Pre-activations,
// biases, accumulations and gradients are FP32; master weights and Adam
// moments are FP32.
#include <math.h>
#include <stdint.h>

#include <algorithm>
#include <new>
#include <string>

#include "../../include/lb.h"
#include "lb_internal.h"

namespace {

using lbk::Geom;
using lbk::wrap_node;

constexpr int D0 = 27, D1 = 64, D2 = 64, D3 = 3;
constexpr int OFF_W1 = 0, OFF_B1 = OFF_W1 + D1 * D0, OFF_W2 = OFF_B1 + D1, OFF_B2 = OFF_W2 + D2 * D1,
              OFF_W3 = OFF_B2 + D2, OFF_B3 = OFF_W3 + D3 * D2, NPARAM = OFF_B3 + D3;
constexpr float FEAT_LENGTH = 4.0f;
constexpr float R_CUT = 8.0f;
constexpr int NNB = 8;

__device__ __forceinline__ float bf16r(float v) { return __bfloat162float(__float2bfloat16_rn(v)); }
__device__ __forceinline__ float silu(float z) { return z / (1.0f + expf(-z)); }

// SiLU of the inference forward, z / (1 + e^-z), from the hardware base-2
// exponential and reciprocal (about 10 instructions against about 25 for
// expf and the IEEE division).  e^-z = 2^t, t = -z log2(e), by Cody and
// Waite's additive range reduction: t_hi = fl(-z L_hi), and the rest
// r = (-z L_hi - t_hi) + (-z) L_lo (the first term exact from an FMA,
// L_hi + L_lo = log2(e) to 2^-50), so 2^t = 2^t_hi (1 + r ln 2) to O(r^2),
// r < 2^-17.  ex2.approx and rcp.approx are each within 2 ulp: the result
// is within a few ulp of z / (1 + e^-z), the class of the library path,
// and the bfloat16 rounding that follows it decides the same way save for
// values within those few ulp of a rounding boundary.  t is clamped at 126
// so that 1 + 2^t stays finite (there z < -87 and z / (1 + e^-z) is below
// 2^-119 in magnitude either way).
__device__ __forceinline__ float silu_fwd(float z) {
    constexpr float L_HI = 1.44269502162933349609375f;  // log2(e) rounded to float
    constexpr float L_LO = 1.925962989091e-8f;        // log2(e) - L_HI
    constexpr float LN2 = 0.693147180559945309f;
    const float t = -z * L_HI;
    const float r = fmaf(-z, L_HI, -t) + (-z) * L_LO;
    float e, q;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(e) : "f"(fminf(t, 126.0f)));
    e = fmaf(e, r * LN2, e);
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(q) : "f"(1.0f + e));
    return z * q;
}
__device__ __forceinline__ float dsilu(float z) {
    const float s = 1.0f / (1.0f + expf(-z));
    return s * (1.0f + z * (1.0f - s));
}

// ------------------------------------------------- tensor-core forward
// The two 64-wide layers on the 5th-generation tensor cores: a CTA of 128
// threads takes tiles of 128 samples; per layer one thread issues
// tcgen05.mma (kind::f16, bfloat16 operands from shared memory, FP32
// accumulator in 64 tensor-memory columns, M = 128, N = 64, K = 16 per
// instruction) and commits to an mbarrier; thread r then reads row r of the
// accumulator (tcgen05.ld) and applies bias and SiLU, rounding to bfloat16
// for the next layer.  The 64 -> 3 output layer runs on the CUDA cores.
//
// Operands use the K-major layout without swizzle: 8 x 16-byte core
// matrices (8 rows of 8 bfloat16), core matrices along K 128 bytes apart
// (leading byte offset), 8-row groups K/8 * 128 bytes apart (stride byte
// offset).
namespace tc {

constexpr int M = 128;          // samples per tile = threads per CTA
constexpr int K1 = 32;          // 27 inputs padded to two K = 16 steps
constexpr int NCOL = 64;        // tensor-memory columns (both layers reuse them)
// shared-memory layout (bytes)
constexpr int B1 = 0;                       // W1 [64][32] bf16
constexpr int B2 = B1 + D1 * K1 * 2;        // W2 [64][64] bf16
constexpr int A2 = B2 + D2 * D1 * 2;        // h1 [128][64] bf16
constexpr int A1 = A2;                      // x  [128][32] bf16, in h1's place: the first
                                            // product has completed before h1 is written,
                                            // the second before the next tile's x
constexpr int W3S = A2 + M * D1 * 2;        // W3 [3][64] float (bf16-rounded)
constexpr int BIAS = W3S + D3 * D2 * 4;     // b1 b2 b3 float
constexpr int MBAR = BIAS + 132 * 4;        // mbarrier (8 bytes)
constexpr int TADDR = MBAR + 8;             // tensor-memory address from tcgen05.alloc
constexpr int USED = TADDR + 8;
// requested dynamic shared memory: it admits at most 7 CTAs per SM (with the
// 1 KB the SM reserves per CTA), so at most 7 x 64 of the 512 tensor-memory
// columns are ever allocated at once (alloc never waits)
constexpr int FWD_CTAS = 7;
constexpr int SMEM = 30 * 1024;
static_assert(USED <= SMEM, "shared layout");
static_assert((FWD_CTAS + 1) * (SMEM + 1024) > 228 * 1024 && FWD_CTAS * NCOL <= 512, "CTAs per SM");

// byte offset of element (row, k) in a K-major no-swizzle operand with K columns
__host__ __device__ constexpr int kmajor_off(int row, int k, int K) {
    return (row >> 3) * (K / 8) * 128 + (k >> 3) * 128 + (row & 7) * 16 + (k & 7) * 2;
}

__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
    return (uint64_t)((addr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);  // version 1, no swizzle
}

// instruction descriptor: D FP32, A and B bfloat16, both K-major, N, M
constexpr uint32_t IDESC = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(D1 >> 3) << 17) | ((uint32_t)(M >> 4) << 24);

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// instruction descriptor for M = 128 and a given N (multiple of 16)
__host__ __device__ constexpr uint32_t idesc_n(int N) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma(uint32_t dtmem, uint64_t a, uint64_t b, uint32_t accumulate,
                                    uint32_t idesc = IDESC) {
    asm volatile(
        "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(dtmem),
        "l"(a), "l"(b), "r"(idesc), "r"(accumulate));
}

__device__ __forceinline__ void commit(uint32_t mbar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar) : "memory");
}

constexpr long long WAIT_POLLS = 1LL << 26;  // default bound of a wait (polls of the mbarrier)

// Bounded wait for phase `parity` of the mbarrier; false on timeout.
__device__ __forceinline__ bool wait_phase(uint32_t mbar, uint32_t parity, long long polls) {
    for (long long it = 0; it < polls; ++it) {
        uint32_t done;
        asm volatile(
            "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(done)
            : "r"(mbar), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}

// 64 consecutive FP32 columns of this thread's accumulator row
__device__ __forceinline__ void load_row64(uint32_t taddr, float (&v)[64]) {
    uint32_t r[64];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x64.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31,%32,%33,%34,%35,%36,%37,%38,%39,"
        "%40,%41,%42,%43,%44,%45,%46,%47,%48,%49,%50,%51,%52,%53,%54,%55,%56,%57,%58,%59,%60,%61,%62,%63}, [%64];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31]),
          "=r"(r[32]), "=r"(r[33]), "=r"(r[34]), "=r"(r[35]), "=r"(r[36]), "=r"(r[37]), "=r"(r[38]), "=r"(r[39]),
          "=r"(r[40]), "=r"(r[41]), "=r"(r[42]), "=r"(r[43]), "=r"(r[44]), "=r"(r[45]), "=r"(r[46]), "=r"(r[47]),
          "=r"(r[48]), "=r"(r[49]), "=r"(r[50]), "=r"(r[51]), "=r"(r[52]), "=r"(r[53]), "=r"(r[54]), "=r"(r[55]),
          "=r"(r[56]), "=r"(r[57]), "=r"(r[58]), "=r"(r[59]), "=r"(r[60]), "=r"(r[61]), "=r"(r[62]), "=r"(r[63])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int k = 0; k < 64; ++k) v[k] = __uint_as_float(r[k]);
}

// 32 and 16 consecutive FP32 columns of this thread's accumulator row
__device__ __forceinline__ void load_row32(uint32_t taddr, float* v) {
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int k = 0; k < 32; ++k) v[k] = __uint_as_float(r[k]);
}

__device__ __forceinline__ void load_row8(uint32_t taddr, float (&v)[8]) {
    uint32_t r[8];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
                 : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int k = 0; k < 8; ++k) v[k] = __uint_as_float(r[k]);
}

__device__ __forceinline__ void load_row16(uint32_t taddr, float* v) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int k = 0; k < 16; ++k) v[k] = __uint_as_float(r[k]);
}

// 64 consecutive FP32 columns of this thread's row into tensor memory
__device__ __forceinline__ void store_row64(uint32_t taddr, const float (&v)[64]) {
    uint32_t r[64];
#pragma unroll
    for (int k = 0; k < 64; ++k) r[k] = __float_as_uint(v[k]);
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x64.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,"
        "%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31,%32,%33,%34,%35,%36,%37,%38,%39,%40,"
        "%41,%42,%43,%44,%45,%46,%47,%48,%49,%50,%51,%52,%53,%54,%55,%56,%57,%58,%59,%60,%61,%62,%63,%64};"
        ::"r"(taddr), "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7]),
          "r"(r[8]), "r"(r[9]), "r"(r[10]), "r"(r[11]), "r"(r[12]), "r"(r[13]), "r"(r[14]), "r"(r[15]),
          "r"(r[16]), "r"(r[17]), "r"(r[18]), "r"(r[19]), "r"(r[20]), "r"(r[21]), "r"(r[22]), "r"(r[23]),
          "r"(r[24]), "r"(r[25]), "r"(r[26]), "r"(r[27]), "r"(r[28]), "r"(r[29]), "r"(r[30]), "r"(r[31]),
          "r"(r[32]), "r"(r[33]), "r"(r[34]), "r"(r[35]), "r"(r[36]), "r"(r[37]), "r"(r[38]), "r"(r[39]),
          "r"(r[40]), "r"(r[41]), "r"(r[42]), "r"(r[43]), "r"(r[44]), "r"(r[45]), "r"(r[46]), "r"(r[47]),
          "r"(r[48]), "r"(r[49]), "r"(r[50]), "r"(r[51]), "r"(r[52]), "r"(r[53]), "r"(r[54]), "r"(r[55]),
          "r"(r[56]), "r"(r[57]), "r"(r[58]), "r"(r[59]), "r"(r[60]), "r"(r[61]), "r"(r[62]), "r"(r[63])
        : "memory");
    asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {  // both rounded to nearest even
    const __nv_bfloat162 p = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<const uint32_t*>(&p);
}

// Transposed write of 2-byte values into a K-major operand whose K runs
// over the 128 samples of a tile: this thread (sample s) holds v[r] for
// rows row0 + r; lane pairs (s, s^1) exchange by shuffle and each writes
// the 32-bit words (samples 2j, 2j + 1) of every other row.
template <int NROWS>
__device__ __forceinline__ void write_transposed(unsigned char* base, int row0, int s, const float* v) {
    const bool odd = (s & 1) != 0;
#pragma unroll
    for (int r = 0; r < NROWS; ++r) {
        const float mine = v[r];
        const float other = __shfl_xor_sync(0xffffffffu, mine, 1);
        if (((r & 1) != 0) == odd) {
            const uint32_t w = odd ? pack_bf16(other, mine) : pack_bf16(mine, other);
            *(uint32_t*)(base + kmajor_off(row0 + r, s & ~1, 128)) = w;
        }
    }
}


}  // namespace tc

// Forward pass on the tensor cores; each wait on the tensor-core pipeline
// polls at most `polls` times.  On a timeout status[0] is set to 1 and the
// kernel stops: it first waits (default bound) for the work it issued, then
// frees its tensor memory.
__global__ void __launch_bounds__(tc::M, tc::FWD_CTAS) km_forward_tc(const float* __restrict__ params, long long n,
                                                       const float* __restrict__ feat, float* __restrict__ out,
                                                       int* __restrict__ status, long long polls) {
    using namespace tc;
    extern __shared__ __align__(1024) unsigned char smem[];
    const int tid = threadIdx.x, warp = tid >> 5;
    const uint32_t mbar = smem_u32(smem + MBAR);
    float* w3 = (float*)(smem + W3S);
    float* bias = (float*)(smem + BIAS);

    // weights, rounded to bfloat16, in the K-major layout; the loops have
    // fixed trip counts and are unrolled so that every load of a thread is
    // in flight at once (a CTA starts with one memory latency, not 50)
    static_assert(D1 * K1 % M == 0 && D2 * D1 % M == 0 && D1 <= M && D2 <= M, "staging loops");
#pragma unroll
    for (int it = 0; it < D1 * K1 / M; ++it) {
        const int i = it * M + tid, r = i / K1, k = i % K1;
        const float w = k < D0 ? params[OFF_W1 + r * D0 + k] : 0.0f;
        *(__nv_bfloat16*)(smem + B1 + kmajor_off(r, k, K1)) = __float2bfloat16_rn(w);
    }
#pragma unroll
    for (int it = 0; it < D2 * D1 / M; ++it) {
        const int i = it * M + tid, r = i / D1, k = i % D1;
        *(__nv_bfloat16*)(smem + B2 + kmajor_off(r, k, D1)) = __float2bfloat16_rn(params[OFF_W2 + i]);
    }
#pragma unroll
    for (int it = 0; it < (D3 * D2 + M - 1) / M; ++it) {
        const int i = it * M + tid;
        if (i < D3 * D2) w3[i] = bf16r(params[OFF_W3 + i]);
    }
    if (tid < D1) bias[tid] = params[OFF_B1 + tid];
    if (tid < D2) bias[D1 + tid] = params[OFF_B2 + tid];
    if (tid < D3) bias[D1 + D2 + tid] = params[OFF_B3 + tid];
    if (tid == 0) asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(mbar) : "memory");
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(smem + TADDR)),
                     "r"(NCOL)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tbase = *(volatile uint32_t*)(smem + TADDR);
    const uint32_t trow = tbase + ((uint32_t)(warp * 32) << 16);  // this warp's 32 lanes
    const uint32_t a1 = smem_u32(smem + A1), a2 = smem_u32(smem + A2);
    const uint32_t b1 = smem_u32(smem + B1), b2 = smem_u32(smem + B2);
    uint32_t phase = 0;
    bool ok = true;

    for (long long t = blockIdx.x; t * M < n && ok; t += gridDim.x) {
        const long long s = t * M + tid;  // this thread's sample
        // x: 27 features rounded to bfloat16, zero-padded to 32
        {
            float x[K1];
#pragma unroll
            for (int k = 0; k < K1; ++k) x[k] = (s < n && k < D0) ? feat[s * D0 + k] : 0.0f;
#pragma unroll
            for (int kg = 0; kg < K1 / 8; ++kg) {
                uint4 v;
                v.x = pack_bf16(x[8 * kg + 0], x[8 * kg + 1]);
                v.y = pack_bf16(x[8 * kg + 2], x[8 * kg + 3]);
                v.z = pack_bf16(x[8 * kg + 4], x[8 * kg + 5]);
                v.w = pack_bf16(x[8 * kg + 6], x[8 * kg + 7]);
                *(uint4*)(smem + A1 + kmajor_off(tid, 8 * kg, K1)) = v;
            }
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncthreads();
        if (tid == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            for (int ks = 0; ks < K1 / 16; ++ks)
                mma(tbase, smem_desc(a1 + ks * 256, 128, (K1 / 8) * 128), smem_desc(b1 + ks * 256, 128, (K1 / 8) * 128),
                    ks > 0);
            commit(mbar);
        }
        ok = __syncthreads_and(wait_phase(mbar, phase, polls));  // uniform across the CTA
        phase ^= 1u;
        if (!ok) break;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        // h1 = bf16(silu(z1 + b1)) into the layer-2 operand, 8 accumulator
        // columns at a time (a rolled loop: few registers, little code)
#pragma unroll 1
        for (int kg = 0; kg < D1 / 8; ++kg) {
            float z[8], h[8];
            load_row8(trow + 8 * kg, z);
#pragma unroll
            for (int e = 0; e < 8; ++e) h[e] = silu_fwd(z[e] + bias[8 * kg + e]);
            uint4 v;
            v.x = pack_bf16(h[0], h[1]);
            v.y = pack_bf16(h[2], h[3]);
            v.z = pack_bf16(h[4], h[5]);
            v.w = pack_bf16(h[6], h[7]);
            *(uint4*)(smem + A2 + kmajor_off(tid, 8 * kg, D1)) = v;
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncthreads();
        if (tid == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            for (int ks = 0; ks < D1 / 16; ++ks)
                mma(tbase, smem_desc(a2 + ks * 256, 128, (D1 / 8) * 128), smem_desc(b2 + ks * 256, 128, (D1 / 8) * 128),
                    ks > 0);
            commit(mbar);
        }
        ok = __syncthreads_and(wait_phase(mbar, phase, polls));
        phase ^= 1u;
        if (!ok) break;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        // h2 = bf16(silu(z2 + b2)); y = W3 h2 + b3 on the CUDA cores, summed
        // over k = 0..63 in order
        float y0 = bias[D1 + D2], y1 = bias[D1 + D2 + 1], y2 = bias[D1 + D2 + 2];
#pragma unroll 1
        for (int kg = 0; kg < D2 / 8; ++kg) {
            float z[8];
            load_row8(trow + 8 * kg, z);
#pragma unroll
            for (int e = 0; e < 8; ++e) {
                const int k = 8 * kg + e;
                const float h = bf16r(silu_fwd(z[e] + bias[D1 + k]));
                y0 = fmaf(h, w3[k], y0);
                y1 = fmaf(h, w3[D2 + k], y1);
                y2 = fmaf(h, w3[2 * D2 + k], y2);
            }
        }
        if (s < n) {
            out[s * D3] = y0;
            out[s * D3 + 1] = y1;
            out[s * D3 + 2] = y2;
        }
        // every thread's accumulator reads are complete before the next tile's MMA
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncthreads();
    }
    if (!ok) {
        if (tid == 0) atomicExch(status, 1);
        wait_phase(mbar, phase ^ 1u, WAIT_POLLS);  // bounded: let the tensor-core work in flight finish
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tbase), "r"(NCOL) : "memory");
}

// ------------------------------------------------ tensor-core training
// Gradient of the mean squared error (1 / 3n) sum (y - t)^2 on the tensor
// cores.  A CTA of 128 threads takes tiles of 128 samples (thread r is
// sample r); per tile, each step a tcgen05.mma (kind::f16, M = 128) with
// its accumulator in tensor memory, committed to an mbarrier:
//   z1 = x W1^T, z2 = h1 W2^T                          (forward, as km_forward_tc)
//   gh1 = gz2 W2  (B = W2^T)                           (N = 64, K = 64)
//   D3 += [h2^T; 1; 0] [gy^T; 0]^T                      (N = 16, K = 128 samples)
//   DG += [gz2^T; gz1^T] [h1^T; x^T; 1; 0]^T            (N = 112, K = 128 samples)
// so that, summed over the CTA's tiles, DG holds dW2 (rows 0-63, columns
// 0-63), dW1 (rows 64-127, columns 64-90), db2 and db1 (column 96), and D3
// holds dW3^T (rows 0-63, columns 0-2) and db3 (row 64); they are added to
// the global gradient once per CTA.  The operands of these products are
// bfloat16: x, h1, h2 (as in the forward) and gy, gz2, gz1 (rounded to
// nearest even); gh2 = gy W3 and the SiLU derivatives are FP32 on the CUDA
// cores.  Operands whose K runs over the samples are written transposed
// into the K-major layout of the forward operands.
namespace tc {
struct G {  // shared memory (bytes)
    static constexpr int B1 = 0;                  // W1   [64][32]   K-major over inputs
    static constexpr int B2 = B1 + 64 * 32 * 2;   // W2   [64][64]   K-major over inputs
    static constexpr int W2T = B2 + 64 * 64 * 2;  // W2^T [64][64]   K-major over outputs
    static constexpr int A1 = W2T + 64 * 64 * 2;  // x    [128][32]
    static constexpr int A2 = A1 + 128 * 32 * 2;  // h1   [128][64]
    static constexpr int GZ = A2 + 128 * 64 * 2;  // gz2  [128][64]
    static constexpr int AG = GZ + 128 * 64 * 2;  // [gz2^T; gz1^T]       [128][128 samples]
    static constexpr int BG = AG + 128 * 128 * 2; // [h1^T; x^T; 1; 0]    [112][128 samples]
    static constexpr int A3 = BG + 112 * 128 * 2; // [h2^T; 1; 0]         [128][128 samples]
    static constexpr int B3 = A3 + 128 * 128 * 2; // [gy^T; 0]            [16][128 samples]
    static constexpr int W3S = B3 + 16 * 128 * 2; // W3 float [3][64] (bfloat16-rounded)
    static constexpr int BIAS = W3S + 3 * 64 * 4; // b1 b2 b3
    static constexpr int MBAR = BIAS + 132 * 4;
    static constexpr int TADDR = MBAR + 8;
    static constexpr int USED = TADDR + 8;
};
constexpr int GSMEM = 200 * 1024;  // one CTA per SM: its 256 tensor-memory columns never wait
static_assert(G::USED <= GSMEM, "training shared layout");
constexpr int GCOLS = 256;
constexpr int TZ = 0, TDG = 64, TD3 = 176, TZ1 = 192;  // tensor-memory columns
constexpr int KS = 128;                                // samples: K of the weight-gradient products
constexpr uint32_t SBO_S = (KS / 8) * 128;             // stride byte offset of those operands

// Before a tensor-core phase: the operands written by the threads become
// visible to the tensor cores, and every thread's tensor-memory reads are
// ordered before the products.
__device__ __forceinline__ void before_issue() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
}
// After issuing and committing: the bounded wait, uniform across the CTA.
__device__ __forceinline__ bool after_issue(uint32_t mbar, uint32_t& phase, long long polls) {
    const bool ok = __syncthreads_and(wait_phase(mbar, phase, polls));
    phase ^= 1u;
    if (ok) asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    return ok;
}
}  // namespace tc

__global__ void __launch_bounds__(tc::M, 1) km_grad_tc(const float* __restrict__ params, long long n,
                                                       const float* __restrict__ feat,
                                                       const float* __restrict__ target, float* __restrict__ grad,
                                                       float* __restrict__ sse, int* __restrict__ status,
                                                       long long polls) {
    using namespace tc;
    extern __shared__ __align__(1024) unsigned char smem[];
    const int tid = threadIdx.x, warp = tid >> 5;
    const uint32_t mbar = smem_u32(smem + G::MBAR);
    float* w3 = (float*)(smem + G::W3S);
    float* bias = (float*)(smem + G::BIAS);
    const float gscale = 2.0f / (3.0f * (float)n);

    // weights (bfloat16) and the constant rows of the gradient operands
    for (int i = tid; i < D1 * K1; i += M) {
        const int r = i / K1, k = i % K1;
        const float w = k < D0 ? params[OFF_W1 + r * D0 + k] : 0.0f;
        *(__nv_bfloat16*)(smem + G::B1 + kmajor_off(r, k, K1)) = __float2bfloat16_rn(w);
    }
    for (int i = tid; i < D2 * D1; i += M) {
        const int o = i / D1, k = i % D1;
        const __nv_bfloat16 w = __float2bfloat16_rn(params[OFF_W2 + i]);
        *(__nv_bfloat16*)(smem + G::B2 + kmajor_off(o, k, D1)) = w;   // [o][i]
        *(__nv_bfloat16*)(smem + G::W2T + kmajor_off(k, o, D2)) = w;  // [i][o]
    }
    for (int i = tid; i < D3 * D2; i += M) w3[i] = bf16r(params[OFF_W3 + i]);
    for (int i = tid; i < D1; i += M) bias[i] = params[OFF_B1 + i];
    for (int i = tid; i < D2; i += M) bias[D1 + i] = params[OFF_B2 + i];
    if (tid < D3) bias[D1 + D2 + tid] = params[OFF_B3 + tid];
    {
        const __nv_bfloat16 one = __float2bfloat16_rn(1.0f), zero = __float2bfloat16_rn(0.0f);
        for (int r = 96; r < 112; ++r)  // BG: the ones row, then zeros
            *(__nv_bfloat16*)(smem + G::BG + kmajor_off(r, tid, KS)) = r == 96 ? one : zero;
        for (int r = 64; r < 128; ++r)  // A3: the ones row, then zeros
            *(__nv_bfloat16*)(smem + G::A3 + kmajor_off(r, tid, KS)) = r == 64 ? one : zero;
        for (int r = 3; r < 16; ++r) *(__nv_bfloat16*)(smem + G::B3 + kmajor_off(r, tid, KS)) = zero;
    }
    if (tid == 0) asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(mbar) : "memory");
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(smem + G::TADDR)),
                     "r"(GCOLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tbase = *(volatile uint32_t*)(smem + G::TADDR);
    const uint32_t lanes = (uint32_t)(warp * 32) << 16;  // this warp's 32 lanes
    const uint32_t a1 = smem_u32(smem + G::A1), a2 = smem_u32(smem + G::A2), gz = smem_u32(smem + G::GZ);
    const uint32_t b1 = smem_u32(smem + G::B1), b2 = smem_u32(smem + G::B2), w2t = smem_u32(smem + G::W2T);
    const uint32_t ag = smem_u32(smem + G::AG), bg = smem_u32(smem + G::BG);
    const uint32_t a3 = smem_u32(smem + G::A3), b3 = smem_u32(smem + G::B3);
    uint32_t phase = 0;
    bool ok = true, first = true;
    float asse = 0.0f;


    for (long long t = blockIdx.x; t * M < n && ok; t += gridDim.x) {
        const long long s = t * M + tid;
        const bool live = s < n;
        float z[64];
        {  // x: bfloat16, zero-padded to 32; also x^T into the gradient operand
            float x[K1];
#pragma unroll
            for (int k = 0; k < K1; ++k) x[k] = (live && k < D0) ? feat[s * D0 + k] : 0.0f;
#pragma unroll
            for (int kg = 0; kg < K1 / 8; ++kg) {
                uint4 v;
                v.x = pack_bf16(x[8 * kg + 0], x[8 * kg + 1]);
                v.y = pack_bf16(x[8 * kg + 2], x[8 * kg + 3]);
                v.z = pack_bf16(x[8 * kg + 4], x[8 * kg + 5]);
                v.w = pack_bf16(x[8 * kg + 6], x[8 * kg + 7]);
                *(uint4*)(smem + G::A1 + kmajor_off(tid, 8 * kg, K1)) = v;
            }
            write_transposed<K1>(smem + G::BG, 64, tid, x);
        }
        before_issue();
        if (tid == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            for (int ks = 0; ks < K1 / 16; ++ks)
                mma(tbase + TZ, smem_desc(a1 + ks * 256, 128, (K1 / 8) * 128), smem_desc(b1 + ks * 256, 128, (K1 / 8) * 128),
                    ks > 0);
            commit(mbar);
        }
        ok = after_issue(mbar, phase, polls);
        if (!ok) break;
        load_row64(tbase + lanes + TZ, z);
        store_row64(tbase + lanes + TZ1, z);  // z1, for the SiLU derivative of the backward pass
        {
            float h[64];
#pragma unroll
            for (int k = 0; k < 64; ++k) h[k] = silu(z[k] + bias[k]);
#pragma unroll
            for (int kg = 0; kg < D1 / 8; ++kg) {
                uint4 v;
                v.x = pack_bf16(h[8 * kg + 0], h[8 * kg + 1]);
                v.y = pack_bf16(h[8 * kg + 2], h[8 * kg + 3]);
                v.z = pack_bf16(h[8 * kg + 4], h[8 * kg + 5]);
                v.w = pack_bf16(h[8 * kg + 6], h[8 * kg + 7]);
                *(uint4*)(smem + G::A2 + kmajor_off(tid, 8 * kg, D1)) = v;
            }
            write_transposed<64>(smem + G::BG, 0, tid, h);
        }
        before_issue();
        if (tid == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            for (int ks = 0; ks < D1 / 16; ++ks)
                mma(tbase + TZ, smem_desc(a2 + ks * 256, 128, (D1 / 8) * 128), smem_desc(b2 + ks * 256, 128, (D1 / 8) * 128),
                    ks > 0);
            commit(mbar);
        }
        ok = after_issue(mbar, phase, polls);
        if (!ok) break;
        load_row64(tbase + lanes + TZ, z);  // z2
        {
            float h[64], gy[D3];  // h holds h2, then gz2
            float y0 = bias[D1 + D2], y1 = bias[D1 + D2 + 1], y2 = bias[D1 + D2 + 2];
#pragma unroll
            for (int k = 0; k < D2; ++k) {
                h[k] = bf16r(silu(z[k] + bias[D1 + k]));
                y0 = fmaf(h[k], w3[k], y0);
                y1 = fmaf(h[k], w3[D2 + k], y1);
                y2 = fmaf(h[k], w3[2 * D2 + k], y2);
            }
            write_transposed<64>(smem + G::A3, 0, tid, h);
            const float yv[3] = {y0, y1, y2};
#pragma unroll
            for (int o = 0; o < D3; ++o) {
                float d = 0.0f;
                if (live) d = yv[o] - target[s * D3 + o];
                asse = fmaf(d, d, asse);
                gy[o] = gscale * d;
            }
            write_transposed<D3>(smem + G::B3, 0, tid, gy);
#pragma unroll
            for (int k = 0; k < D2; ++k) {
                const float g = fmaf(gy[0], w3[k], fmaf(gy[1], w3[D2 + k], gy[2] * w3[2 * D2 + k]));
                h[k] = g * dsilu(z[k] + bias[D1 + k]);
            }
#pragma unroll
            for (int kg = 0; kg < D2 / 8; ++kg) {
                uint4 v;
                v.x = pack_bf16(h[8 * kg + 0], h[8 * kg + 1]);
                v.y = pack_bf16(h[8 * kg + 2], h[8 * kg + 3]);
                v.z = pack_bf16(h[8 * kg + 4], h[8 * kg + 5]);
                v.w = pack_bf16(h[8 * kg + 6], h[8 * kg + 7]);
                *(uint4*)(smem + G::GZ + kmajor_off(tid, 8 * kg, D2)) = v;
            }
            write_transposed<64>(smem + G::AG, 0, tid, h);
        }
        const bool acc = !first;
        before_issue();
        if (tid == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            for (int ks = 0; ks < D2 / 16; ++ks)  // gh1 = gz2 W2
                mma(tbase + TZ, smem_desc(gz + ks * 256, 128, (D2 / 8) * 128), smem_desc(w2t + ks * 256, 128, (D2 / 8) * 128),
                    ks > 0);
            for (int ks = 0; ks < KS / 16; ++ks)  // D3 += [h2^T; 1] [gy^T]^T
                mma(tbase + TD3, smem_desc(a3 + ks * 256, 128, SBO_S), smem_desc(b3 + ks * 256, 128, SBO_S),
                    acc || ks > 0, idesc_n(16));
            commit(mbar);
        }
        ok = after_issue(mbar, phase, polls);
        if (!ok) break;
        {
            float gh[64];
            load_row64(tbase + lanes + TZ, gh);
            load_row64(tbase + lanes + TZ1, z);  // z1
#pragma unroll
            for (int k = 0; k < D1; ++k) gh[k] *= dsilu(z[k] + bias[k]);
            write_transposed<64>(smem + G::AG, 64, tid, gh);
        }
        before_issue();
        if (tid == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            for (int ks = 0; ks < KS / 16; ++ks)  // DG += [gz2^T; gz1^T] [h1^T; x^T; 1]^T
                mma(tbase + TDG, smem_desc(ag + ks * 256, 128, SBO_S), smem_desc(bg + ks * 256, 128, SBO_S),
                    acc || ks > 0, idesc_n(112));
            commit(mbar);
        }
        ok = after_issue(mbar, phase, polls);
        first = false;
        // every thread's tensor-memory reads are complete before the next tile's products
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncthreads();
    }
    if (!ok) {
        if (tid == 0) atomicExch(status, 1);
        wait_phase(mbar, phase ^ 1u, WAIT_POLLS);  // bounded: let the tensor-core work in flight finish
    } else if (!first) {  // this CTA's gradient sums into the global gradient
        float v[64];
        load_row64(tbase + lanes + TDG, v);
        float u[32];
        load_row32(tbase + lanes + TDG + 64, u);
        float w[16];
        load_row16(tbase + lanes + TDG + 96, w);
        float d3[16];
        load_row16(tbase + lanes + TD3, d3);
        if (tid < 64) {
            for (int c = 0; c < D1; ++c) atomicAdd(&grad[OFF_W2 + tid * D1 + c], v[c]);
            atomicAdd(&grad[OFF_B2 + tid], w[0]);
            for (int k = 0; k < D3; ++k) atomicAdd(&grad[OFF_W3 + k * D2 + tid], d3[k]);
        } else {
            const int o = tid - 64;
            for (int c = 0; c < D0; ++c) atomicAdd(&grad[OFF_W1 + o * D0 + c], u[c]);
            atomicAdd(&grad[OFF_B1 + o], w[0]);
            if (tid == 64)
                for (int k = 0; k < D3; ++k) atomicAdd(&grad[OFF_B3 + k], d3[k]);
        }
    }
    for (int off = 16; off > 0; off >>= 1) asse += __shfl_xor_sync(0xffffffffu, asse, off);
    if ((tid & 31) == 0) atomicAdd(sse, asse);
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tbase), "r"(GCOLS) : "memory");
}

// Minibatch s of lb_mlp_train: sample b takes row j = h(seed, s, b) mod n of
// (feat, target), h the SplitMix64 finaliser (Steele, Lea and Flood, 2014)
// of seed + (s * batch + b + 1) * golden-ratio constant, shifted right by 11;
// targets divided by their scale.  One thread a sample.
__device__ __forceinline__ unsigned long long splitmix64(unsigned long long x) {
    x ^= x >> 30;
    x *= 0xBF58476D1CE4E5B9ull;
    x ^= x >> 27;
    x *= 0x94D049BB133111EBull;
    return x ^ (x >> 31);
}

__global__ void km_gather(unsigned long long seed, long long s, int batch, long long n, const float* __restrict__ feat,
                          const float* __restrict__ target, float inv_scale, float* __restrict__ bfeat,
                          float* __restrict__ btarget) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= batch) return;
    const unsigned long long c = (unsigned long long)s * (unsigned long long)batch + (unsigned long long)b + 1ull;
    const long long j = (long long)((splitmix64(seed + c * 0x9E3779B97F4A7C15ull) >> 11) % (unsigned long long)n);
#pragma unroll
    for (int k = 0; k < D0; ++k) bfeat[(long long)b * D0 + k] = feat[j * D0 + k];
#pragma unroll
    for (int a = 0; a < D3; ++a) btarget[(long long)b * D3 + a] = target[j * D3 + a] * inv_scale;
}

// The minibatch's mean squared error into slot k of the loss record.
__global__ void km_record_loss(const float* __restrict__ sse, float inv_count, float* __restrict__ rec, int k) {
    rec[k] = sse[0] * inv_count;
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
// Cell list with cells wider than R_CUT by 1/64 (nc = floor(box / (R_CUT +
// 1/64)) per axis, at least 1), so that the 27 cells around a point's cell
// hold every other point whose float32 separation is within R_CUT: the
// float rounding of a position or of the cell arithmetic (below 1e-3 for
// boxes under 2^16) stays far inside the 1/64.
constexpr float CELL_W = R_CUT + 1.0f / 64.0f;

__device__ __forceinline__ int cell_of(float X, float inv_w, int nc) {
    const int c = (int)(X * inv_w);
    return c < 0 ? 0 : (c >= nc ? nc - 1 : c);
}

// Each point's cell, and its float32 position (round to nearest) with its
// index in w: the neighbour search reads only these.
__global__ void kf_count(const double* __restrict__ pos, long long n, float3 inv_w, int3 nc, int* __restrict__ count,
                         int* __restrict__ cell, float4* __restrict__ fpos) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float x = (float)pos[3 * i], y = (float)pos[3 * i + 1], z = (float)pos[3 * i + 2];
    const int c = (cell_of(z, inv_w.z, nc.z) * nc.y + cell_of(y, inv_w.y, nc.y)) * nc.x + cell_of(x, inv_w.x, nc.x);
    cell[i] = c;
    fpos[i] = make_float4(x, y, z, __int_as_float((int)i));
    atomicAdd(&count[c], 1);
}

// The points in cell order (float4 records as kf_count made them).
__global__ void kf_fill(long long n, const int* __restrict__ cell, const float4* __restrict__ fpos,
                        const int* __restrict__ start, int* __restrict__ cursor, float4* __restrict__ spos) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int c = cell[i];
    spos[start[c] + atomicAdd(&cursor[c], 1)] = fpos[i];
}

// Minimum-image float32 difference along one axis, each operation rounded
// once: d = xj - xi, then d - box above box/2, d + box below -box/2.
__device__ __forceinline__ float min_image_f(float xj, float xi, float box, float half) {
    const float d = __fsub_rn(xj, xi);
    return d > half ? __fsub_rn(d, box) : (d < -half ? __fadd_rn(d, box) : d);
}

// 27 features per point: the fractional offset, then the 8 nearest others
// within R_CUT (minimum image), nearest first, equal distances by lower
// index.  The distances that select and order them are float32, each
// operation rounded once (the definition the oracle states), so one pass
// over the candidates decides exactly: the key of a candidate is the bit
// pattern of its squared distance (non-negative floats order as their bit
// patterns) above its index, kept in an 8-entry insertion list.  One thread
// per point, the points taken in cell order so that a warp's threads walk
// the same cells.
constexpr int KNN_THREADS = 128;

// Offsets -1, 0, 1 of a cell coordinate along an axis with n cells, wrapped
// (every cell once when n < 3): the k-th of count() of them.
struct AxisWalk {
    int c, n;
    __device__ AxisWalk(int c_, int n_) : c(c_), n(n_) {}
    __device__ int count() const { return n >= 3 ? 3 : n; }
    __device__ int at(int k) const {
        if (n < 3) return k;
        const int r = c + k - 1;
        return r < 0 ? r + n : (r >= n ? r - n : r);
    }
};

__global__ void __launch_bounds__(KNN_THREADS)
kf_knn(const double* __restrict__ pos, long long n, Geom g, int3 nc, const int* __restrict__ start,
       const int* __restrict__ cell, const float4* __restrict__ spos, float* __restrict__ feat) {
    const long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= n) return;
    const float4 me = spos[q];
    const int i = __float_as_int(me.w);
    const float box[3] = {(float)g.nx, (float)g.ny, (float)g.nz};
    const float half[3] = {0.5f * box[0], 0.5f * box[1], 0.5f * box[2]};
    const float rc2 = R_CUT * R_CUT;
    unsigned long long bk[NNB];  // (r2 bits << 32) | index, ascending
    int bs[NNB];                 // slot of each in cell order
#pragma unroll
    for (int k = 0; k < NNB; ++k) {
        bk[k] = ~0ull;
        bs[k] = -1;
    }
    const auto consider = [&](int qq) {
        const float4 o = __ldg(spos + qq);
        const float dx = min_image_f(o.x, me.x, box[0], half[0]);
        const float dy = min_image_f(o.y, me.y, box[1], half[1]);
        const float dz = min_image_f(o.z, me.z, box[2], half[2]);
        const float r2 = __fadd_rn(__fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy)), __fmul_rn(dz, dz));
        unsigned long long ck = ((unsigned long long)__float_as_uint(r2) << 32) | (unsigned)__float_as_int(o.w);
        if (!(r2 <= rc2) || qq == q || ck >= bk[NNB - 1]) return;
        int cs = qq;
#pragma unroll
        for (int k = 0; k < NNB; ++k) {
            const bool lt = ck < bk[k];
            const unsigned long long tk = bk[k];
            const int ts = bs[k];
            bk[k] = lt ? ck : tk;
            bs[k] = lt ? cs : ts;
            ck = lt ? tk : ck;
            cs = lt ? ts : cs;
        }
    };
    // the cells around the point's cell, row by row: along x the (up to) 3
    // cells of a row are contiguous in cell order unless the row wraps
    const int c0 = cell[i];
    const int cx = c0 % nc.x, cyz = c0 / nc.x;
    const AxisWalk wy(cyz % nc.y, nc.y), wz(cyz / nc.y, nc.z);
    int xa, xb, xc, xd;  // x cells [xa, xb) and [xc, xd) of every row
    if (nc.x < 3) {
        xa = 0, xb = nc.x, xc = xd = 0;
    } else if (cx == 0) {
        xa = 0, xb = 2, xc = nc.x - 1, xd = nc.x;
    } else if (cx == nc.x - 1) {
        xa = cx - 1, xb = nc.x, xc = 0, xd = 1;
    } else {
        xa = cx - 1, xb = cx + 2, xc = xd = 0;
    }
    for (int kz = 0; kz < wz.count(); ++kz) {
        const int rz = wz.at(kz) * nc.y;
        for (int ky = 0; ky < wy.count(); ++ky) {
            const int row = (rz + wy.at(ky)) * nc.x;
            for (int qq = start[row + xa], e = start[row + xb]; qq < e; ++qq) consider(qq);
            for (int qq = start[row + xc], e = start[row + xd]; qq < e; ++qq) consider(qq);
        }
    }
    float* f = feat + (long long)i * D0;
    for (int a = 0; a < 3; ++a) f[a] = (float)(pos[3 * (long long)i + a] - floor(pos[3 * (long long)i + a]));
    // the vectors: the same float32 differences, exactly scaled by 1/4
#pragma unroll
    for (int k = 0; k < NNB; ++k) {
        float d[3] = {0.0f, 0.0f, 0.0f};
        if (bs[k] >= 0) {
            const float4 o = spos[bs[k]];
            d[0] = min_image_f(o.x, me.x, box[0], half[0]);
            d[1] = min_image_f(o.y, me.y, box[1], half[1]);
            d[2] = min_image_f(o.z, me.z, box[2], half[2]);
        }
        for (int a = 0; a < 3; ++a) f[3 + 3 * k + a] = d[a] * (1.0f / FEAT_LENGTH);
    }
}

// ------------------------------------------- features with a Verlet list
// The same features for a lattice's colloids step after step.  Positions
// move far less than a lattice spacing per step, so the candidates of a
// point are kept from one rebuild to the next.  Let MOVE bound how far any
// point has moved since the rebuild (float32 displacement, minimum image;
// a larger one raises the rebuild flag), so that the distance of any pair
// has changed by at most 2 MOVE (exact distances obey the triangle
// inequality of the periodic box; the float32 ones differ from them by far
// less than 1/64 in boxes below 2^12).  Then the kept candidates of a
// point p are the others within
//   r_in = min(e8 + 4 MOVE + 1/16, R_CUT + SKIN)
// at the rebuild, e8 the 8th smallest distance of another point within
// R_CUT + SKIN (all of them when there are fewer than 8): the 8 points
// nearest at the rebuild are now within e8 + 2 MOVE, so a point beyond r_in
// at the rebuild is now farther than all 8 and is not selected; and if one
// of those 8 is now beyond R_CUT, then e8 > R_CUT - 2 MOVE and r_in reaches
// R_CUT + SKIN >= R_CUT + 2 MOVE, which holds every point now within
// R_CUT.  Selection and ordering then run over the kept candidates with
// the current positions, exactly as over all points.  The rebuild kernels
// run every step but return at once unless the displacement check of the
// step raised the flag.
constexpr float SKIN = 0.125f;  // 0.25 and 0.375 measured 3 and 5 us slower a step (2e5 colloids)
constexpr float MOVE = 0.5f * SKIN - 1.0f / 64.0f;
constexpr float INNER = 4.0f * MOVE + 1.0f / 16.0f;
constexpr float LIST_R = R_CUT + SKIN;
constexpr float CELL_WV = LIST_R + 1.0f / 64.0f;
constexpr float LIST_R2 = LIST_R * LIST_R;
constexpr float MOVE_R2 = MOVE * MOVE;

struct Verlet {
    float4* fnow;    // current float32 position and index (.w), point order
    float4* fbuild;  // position at the last rebuild, point order
    float4* spos;    // positions at the last rebuild in cell order (index in .w)
    int* cell;       // cell of each point at the last rebuild
    int* len;        // candidates of cell-order slot q (-1: more than cap; scan the cells)
    int* list;       // candidate k of slot q at list[k * n + q] (point indices)
    int* count;      // per cell; zero between rebuilds
    int* cursor;     // per cell; zero between rebuilds
    int* start;      // m + 1 cell starts of the last rebuild
    int* flag;       // 1: rebuild this step
    long long n, m;
    int cap;
    int3 nc;
};

// Current float32 positions; raise the flag where a point moved too far.
__global__ void kv_prep(const double* __restrict__ pos, Verlet v, Geom g) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= v.n) return;
    const float x = (float)pos[3 * i], y = (float)pos[3 * i + 1], z = (float)pos[3 * i + 2];
    v.fnow[i] = make_float4(x, y, z, __int_as_float((int)i));
    const float4 b = v.fbuild[i];
    const float bx = (float)g.nx, by = (float)g.ny, bz = (float)g.nz;
    const float dx = min_image_f(x, b.x, bx, 0.5f * bx), dy = min_image_f(y, b.y, by, 0.5f * by),
                dz = min_image_f(z, b.z, bz, 0.5f * bz);
    if (!(dx * dx + dy * dy + dz * dz <= MOVE_R2)) *v.flag = 1;  // also for a first or non-finite build
}

__global__ void kv_count(Verlet v, float3 inv_w) {
    if (!*v.flag) return;
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= v.n) return;
    const float4 p = v.fnow[i];
    const int c = (cell_of(p.z, inv_w.z, v.nc.z) * v.nc.y + cell_of(p.y, inv_w.y, v.nc.y)) * v.nc.x +
                  cell_of(p.x, inv_w.x, v.nc.x);
    v.cell[i] = c;
    atomicAdd(&v.count[c], 1);
}

// Exclusive scan of the m cell counts into start[0..m] by one block: each
// thread sums a contiguous chunk, the block scans the chunk sums.
constexpr int VSCAN_THREADS = 1024;
__global__ void __launch_bounds__(VSCAN_THREADS) kv_scan(Verlet v) {
    if (!*v.flag) return;
    __shared__ int wsum[VSCAN_THREADS / 32];
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    const long long per = (v.m + VSCAN_THREADS - 1) / VSCAN_THREADS;
    const long long a = min(v.m, (long long)t * per), b = min(v.m, a + per);
    int s = 0;
    for (long long c = a; c < b; ++c) s += v.count[c];
    int incl = s;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int u = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += u;
    }
    if (lane == 31) wsum[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        const int w = wsum[lane];
        int wi = w;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int u = __shfl_up_sync(0xffffffffu, wi, o);
            if (lane >= o) wi += u;
        }
        wsum[lane] = wi - w;
    }
    __syncthreads();
    int run = wsum[warp] + incl - s;
    for (long long c = a; c < b; ++c) {
        v.start[c] = run;
        run += v.count[c];
    }
    if (t == VSCAN_THREADS - 1) v.start[v.m] = run;  // the last chunk ends at m
}

__global__ void kv_fill(Verlet v) {
    if (!*v.flag) return;
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= v.n) return;
    const int c = v.cell[i];
    const float4 p = v.fnow[i];
    v.spos[v.start[c] + atomicAdd(&v.cursor[c], 1)] = p;
    v.fbuild[i] = p;
}

// Walk the 27 cells (fewer when an axis has under 3) around cell c0 of the
// last rebuild, calling visit(slot) for every cell-order slot in them.
template <typename Visit>
__device__ __forceinline__ void walk_cells(const Verlet& v, int c0, Visit&& visit) {
    const int cx = c0 % v.nc.x, cyz = c0 / v.nc.x;
    const AxisWalk wy(cyz % v.nc.y, v.nc.y), wz(cyz / v.nc.y, v.nc.z);
    int xa, xb, xc, xd;  // x cells [xa, xb) and [xc, xd) of every row
    if (v.nc.x < 3) {
        xa = 0, xb = v.nc.x, xc = xd = 0;
    } else if (cx == 0) {
        xa = 0, xb = 2, xc = v.nc.x - 1, xd = v.nc.x;
    } else if (cx == v.nc.x - 1) {
        xa = cx - 1, xb = v.nc.x, xc = 0, xd = 1;
    } else {
        xa = cx - 1, xb = cx + 2, xc = xd = 0;
    }
    for (int kz = 0; kz < wz.count(); ++kz) {
        const int rz = wz.at(kz) * v.nc.y;
        for (int ky = 0; ky < wy.count(); ++ky) {
            const int row = (rz + wy.at(ky)) * v.nc.x;
            for (int qq = v.start[row + xa], e = v.start[row + xb]; qq < e; ++qq) visit(qq);
            for (int qq = v.start[row + xc], e = v.start[row + xd]; qq < e; ++qq) visit(qq);
        }
    }
}

// The kept candidates of every cell-order slot (two walks over the cells:
// the 8 smallest distances give r_in, then the points within it are
// listed); then the per-cell counters are cleared for the next rebuild
// (nothing here reads them).
__global__ void __launch_bounds__(KNN_THREADS) kv_build(Verlet v, Geom g) {
    if (!*v.flag) return;
    const long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    for (long long c = tid; c < v.m; c += (long long)gridDim.x * blockDim.x) {
        v.count[c] = 0;
        v.cursor[c] = 0;
    }
    const long long q = tid;
    if (q >= v.n) return;
    const float4 me = v.spos[q];
    const float box[3] = {(float)g.nx, (float)g.ny, (float)g.nz};
    const float half[3] = {0.5f * box[0], 0.5f * box[1], 0.5f * box[2]};
    const auto dist2 = [&](int qq) {
        const float4 o = v.spos[qq];
        const float dx = min_image_f(o.x, me.x, box[0], half[0]);
        const float dy = min_image_f(o.y, me.y, box[1], half[1]);
        const float dz = min_image_f(o.z, me.z, box[2], half[2]);
        return dx * dx + dy * dy + dz * dz;
    };
    const int c0 = v.cell[__float_as_int(me.w)];
    float near[NNB];  // the 8 smallest squared distances within LIST_R, ascending
#pragma unroll
    for (int k = 0; k < NNB; ++k) near[k] = INFINITY;
    walk_cells(v, c0, [&](int qq) {
        if (qq == q) return;
        float r2 = dist2(qq);
        if (!(r2 <= LIST_R2) || r2 >= near[NNB - 1]) return;
#pragma unroll
        for (int k = 0; k < NNB; ++k) {
            const float t = near[k];
            near[k] = fminf(r2, t);
            r2 = fmaxf(r2, t);
        }
    });
    const float r_in = near[NNB - 1] <= LIST_R2 ? fminf(sqrtf(near[NNB - 1]) + INNER, LIST_R) : LIST_R;
    const float r_in2 = r_in * r_in;
    int cnt = 0;
    walk_cells(v, c0, [&](int qq) {
        if (qq == q || !(dist2(qq) <= r_in2)) return;
        if (cnt < v.cap) v.list[(long long)cnt * v.n + q] = __float_as_int(v.spos[qq].w);
        ++cnt;
    });
    v.len[q] = cnt <= v.cap ? cnt : -1;
}

// The 27 features of every point from its kept candidates at their current
// positions (key, order and vectors as kf_knn); a slot whose candidates
// overflowed the list walks the cells of the last rebuild instead.  Clears
// the rebuild flag for the next step.
__global__ void __launch_bounds__(KNN_THREADS)
kv_knn(const double* __restrict__ pos, Verlet v, Geom g, float* __restrict__ feat) {
    const long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (q == 0) *v.flag = 0;
    if (q >= v.n) return;
    const int i = __float_as_int(v.spos[q].w);
    const float4 me = v.fnow[i];
    const float box[3] = {(float)g.nx, (float)g.ny, (float)g.nz};
    const float half[3] = {0.5f * box[0], 0.5f * box[1], 0.5f * box[2]};
    const float rc2 = R_CUT * R_CUT;
    unsigned long long bk[NNB];  // (r2 bits << 32) | index, ascending
#pragma unroll
    for (int k = 0; k < NNB; ++k) bk[k] = ~0ull;
    const auto consider_at = [&](const float4& o, int j) {
        const float dx = min_image_f(o.x, me.x, box[0], half[0]);
        const float dy = min_image_f(o.y, me.y, box[1], half[1]);
        const float dz = min_image_f(o.z, me.z, box[2], half[2]);
        const float r2 = __fadd_rn(__fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy)), __fmul_rn(dz, dz));
        unsigned long long ck = ((unsigned long long)__float_as_uint(r2) << 32) | (unsigned)j;
        if (!(r2 <= rc2) || ck >= bk[NNB - 1]) return;
#pragma unroll
        for (int k = 0; k < NNB; ++k) {
            const bool lt = ck < bk[k];
            const unsigned long long tk = bk[k];
            bk[k] = lt ? ck : tk;
            ck = lt ? tk : ck;
        }
    };
    const int len = v.len[q];
    if (len >= 0) {
        // eight candidates at a time: their indices, then their positions,
        // each batch of loads in flight together
        const int* l = v.list + q;
        for (int k0 = 0; k0 < len; k0 += 8) {
            int j[8];
            float4 o[8];
#pragma unroll
            for (int e = 0; e < 8; ++e) j[e] = k0 + e < len ? __ldg(l + (long long)(k0 + e) * v.n) : -1;
#pragma unroll
            for (int e = 0; e < 8; ++e)
                if (j[e] >= 0) o[e] = __ldg(v.fnow + j[e]);
#pragma unroll
            for (int e = 0; e < 8; ++e)
                if (j[e] >= 0) consider_at(o[e], j[e]);
        }
    } else {
        walk_cells(v, v.cell[i], [&](int qq) {
            const int j = __float_as_int(v.spos[qq].w);
            if (j != i) consider_at(__ldg(v.fnow + j), j);
        });
    }
    float* f = feat + (long long)i * D0;
    for (int a = 0; a < 3; ++a) f[a] = (float)(pos[3 * (long long)i + a] - floor(pos[3 * (long long)i + a]));
#pragma unroll
    for (int k = 0; k < NNB; ++k) {
        float d[3] = {0.0f, 0.0f, 0.0f};
        if (bk[k] != ~0ull) {
            const float4 o = v.fnow[(int)(unsigned)(bk[k] & 0xffffffffull)];
            d[0] = min_image_f(o.x, me.x, box[0], half[0]);
            d[1] = min_image_f(o.y, me.y, box[1], half[1]);
            d[2] = min_image_f(o.z, me.z, box[2], half[2]);
        }
        for (int a = 0; a < 3; ++a) f[3 + 3 * k + a] = d[a] * (1.0f / FEAT_LENGTH);
    }
}

}  // namespace

struct lb_mlp {
    cudaStream_t stream;
    float *p, *g, *m, *v, *sse;
    int* status;              // set by the tensor-core forward kernel on a timed-out wait
    long long wait_polls;     // bound of the tensor-core kernels' waits
    long long t;              // Adam steps taken
    int *ws;                  // feature workspace (cell lists), grown on demand
    size_t ws_ints;
    float* mb;                // lb_mlp_train: minibatch features and targets, then the loss record
    size_t mb_floats;
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

// Wait for the network's stream and report a timed-out tensor-core wait.
lb_status check_status(lb_mlp* net) {
    int st = 0;
    LB_MCUDA(cudaMemcpyAsync(&st, net->status, sizeof(int), cudaMemcpyDeviceToHost, net->stream), "status read");
    LB_MCUDA(cudaStreamSynchronize(net->stream), "stream synchronize");
    if (st) {
        LB_MCUDA(cudaMemsetAsync(net->status, 0, sizeof(int), net->stream), "status reset");
        return mfail(net, LB_ERR_TIMEOUT, "forward kernel: a tensor-core wait timed out");
    }
    return LB_OK;
}


}  // namespace

namespace lbk {

static int3 feature_cells(const int box[3]) {
    int3 nc;
    nc.x = std::max(1, (int)((float)box[0] / CELL_W));
    nc.y = std::max(1, (int)((float)box[1] / CELL_W));
    nc.z = std::max(1, (int)((float)box[2] / CELL_W));
    return nc;
}

// Workspace in ints: the float4 records in point order and in cell order
// (4 n each, first, so 16-byte aligned), count, cursor, start (m + 1), the
// cell of every point, the scan's tile sums.
size_t mlp_features_ws_ints(long long n, const int box[3]) {
    const int3 nc = feature_cells(box);
    const long long m = (long long)nc.x * nc.y * nc.z;
    return (size_t)(8 * n + 3 * m + 1 + n) + scan_ws_ints(m);
}

cudaError_t mlp_features(long long n, const double* pos, const int box[3], float* feat, int* ws, cudaStream_t st) {
    const int3 nc = feature_cells(box);
    const long long m = (long long)nc.x * nc.y * nc.z;
    float4* fpos = (float4*)ws;
    float4* spos = fpos + n;
    int* count = ws + 8 * n;
    int* cursor = count + m;
    int* start = cursor + m;
    int* cell = start + m + 1;
    int* bsum = cell + n;
    Geom g{};
    g.nx = box[0];
    g.ny = box[1];
    g.nz = box[2];
    if (n == 0) return cudaSuccess;
    cudaError_t e = cudaMemsetAsync(count, 0, sizeof(int) * 2 * m, st);
    if (e != cudaSuccess) return e;
    const float3 inv_w = make_float3((float)nc.x / (float)box[0], (float)nc.y / (float)box[1], (float)nc.z / (float)box[2]);
    const unsigned blocks = (unsigned)((n + 255) / 256);
    kf_count<<<blocks, 256, 0, st>>>(pos, n, inv_w, nc, count, cell, fpos);
    e = scan_exclusive(count, m, start, bsum, st);
    if (e != cudaSuccess) return e;
    kf_fill<<<blocks, 256, 0, st>>>(n, cell, fpos, start, cursor, spos);
    kf_knn<<<(unsigned)((n + KNN_THREADS - 1) / KNN_THREADS), KNN_THREADS, 0, st>>>(pos, n, g, nc, start, cell, spos,
                                                                                  feat);
    return cudaGetLastError();
}

static int3 verlet_cells(const int box[3]) {
    int3 nc;
    nc.x = std::max(1, (int)((float)box[0] / CELL_WV));
    nc.y = std::max(1, (int)((float)box[1] / CELL_WV));
    nc.z = std::max(1, (int)((float)box[2] / CELL_WV));
    return nc;
}

int verlet_capacity(long long n, const int box[3]) {
    // mean candidates of a uniform arrangement, plus six standard deviations
    // of a Poisson count and a margin; fuller slots walk the cells
    const double vol = (double)box[0] * box[1] * box[2];
    const double r = LIST_R;
    const double mu = (double)std::max<long long>(n - 1, 0) * (4.0 / 3.0) * 3.14159265358979 * r * r * r / vol;
    const int cap = (int)(mu + 6.0 * sqrt(mu) + 16.0);
    return std::min(512, std::max(32, (cap + 7) / 8 * 8));
}

static size_t up16(size_t b) { return (b + 15) / 16 * 16; }

size_t verlet_ws_bytes(long long n, const int box[3], int cap) {
    const int3 nc = verlet_cells(box);
    const size_t m = (size_t)nc.x * nc.y * nc.z, N = (size_t)n;
    return 3 * up16(16 * N) + 2 * up16(4 * N) + up16(4 * N * (size_t)cap) + 2 * up16(4 * m) + up16(4 * (m + 1)) + 16;
}

static Verlet verlet_view(void* ws, long long n, const int box[3], int cap) {
    Verlet v;
    const int3 nc = verlet_cells(box);
    const size_t m = (size_t)nc.x * nc.y * nc.z, N = (size_t)n;
    char* p = (char*)ws;
    v.fnow = (float4*)p;
    p += up16(16 * N);
    v.fbuild = (float4*)p;
    p += up16(16 * N);
    v.spos = (float4*)p;
    p += up16(16 * N);
    v.cell = (int*)p;
    p += up16(4 * N);
    v.len = (int*)p;
    p += up16(4 * N);
    v.list = (int*)p;
    p += up16(4 * N * (size_t)cap);
    v.count = (int*)p;
    p += up16(4 * m);
    v.cursor = (int*)p;
    p += up16(4 * m);
    v.start = (int*)p;
    p += up16(4 * (m + 1));
    v.flag = (int*)p;
    v.n = n;
    v.m = (long long)m;
    v.cap = cap;
    v.nc = nc;
    return v;
}

cudaError_t verlet_reset(void* ws, long long n, const int box[3], int cap, cudaStream_t st) {
    const Verlet v = verlet_view(ws, n, box, cap);
    cudaError_t e = cudaMemsetAsync(v.count, 0, sizeof(int) * (size_t)v.m, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(v.cursor, 0, sizeof(int) * (size_t)v.m, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(v.flag, 0xff, sizeof(int), st);  // nonzero: rebuild
    return e;
}

cudaError_t verlet_features(void* ws, long long n, int cap, const double* pos, const int box[3], float* feat,
                            cudaStream_t st) {
    if (n == 0) return cudaSuccess;
    const Verlet v = verlet_view(ws, n, box, cap);
    Geom g{};
    g.nx = box[0];
    g.ny = box[1];
    g.nz = box[2];
    const float3 inv_w = make_float3((float)v.nc.x / (float)box[0], (float)v.nc.y / (float)box[1],
                                     (float)v.nc.z / (float)box[2]);
    const unsigned blocks = (unsigned)((n + 255) / 256);
    const unsigned kblocks = (unsigned)((n + KNN_THREADS - 1) / KNN_THREADS);
    kv_prep<<<blocks, 256, 0, st>>>(pos, v, g);
    kv_count<<<blocks, 256, 0, st>>>(v, inv_w);
    kv_scan<<<1, VSCAN_THREADS, 0, st>>>(v);
    kv_fill<<<blocks, 256, 0, st>>>(v);
    kv_build<<<kblocks, KNN_THREADS, 0, st>>>(v, g);
    kv_knn<<<kblocks, KNN_THREADS, 0, st>>>(pos, v, g, feat);
    return cudaGetLastError();
}

cudaError_t mlp_forward(const lb_mlp* net, long long n, const float* feat, float* out, cudaStream_t st) {
    const long long tiles = (n + tc::M - 1) / tc::M;
    const unsigned grid = (unsigned)std::max<long long>(1, std::min<long long>(tiles, 152LL * tc::FWD_CTAS));
    km_forward_tc<<<grid, tc::M, tc::SMEM, st>>>(net->p, n, feat, out, net->status, net->wait_polls);
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
    net->wait_polls = tc::WAIT_POLLS;
    cudaError_t e = cudaMalloc(&net->p, sizeof(float) * (4 * NPARAM + 1));
    if (e == cudaSuccess) {
        net->g = net->p + NPARAM;
        net->m = net->g + NPARAM;
        net->v = net->m + NPARAM;
        net->sse = net->v + NPARAM;
        e = cudaMemsetAsync(net->p, 0, sizeof(float) * (4 * NPARAM + 1), net->stream);
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(net->p, init, sizeof(float) * NPARAM, cudaMemcpyDefault, net->stream);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(km_grad_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, tc::GSMEM);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(km_forward_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, tc::SMEM);
    if (e == cudaSuccess) e = cudaMalloc(&net->status, sizeof(int));
    if (e == cudaSuccess) e = cudaMemsetAsync(net->status, 0, sizeof(int), net->stream);
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
    cudaFree(net->mb);
    cudaFree(net->status);
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

lb_status lb_mlp_set_wait_limit(lb_mlp* net, long long polls) {
    if (!net) return LB_ERR_ARG;
    if (polls < 0) return mfail(net, LB_ERR_ARG, "lb_mlp_set_wait_limit: polls < 0");
    net->wait_polls = polls;
    return LB_OK;
}

lb_status lb_mlp_forward(lb_mlp* net, long long n, const float* feat, float* out) {
    if (!net || n < 0 || (n && (!feat || !out))) return mfail(net, LB_ERR_ARG, "lb_mlp_forward: bad argument");
    if (n == 0) return LB_OK;
    LB_MCUDA(lbk::mlp_forward(net, n, feat, out, net->stream), "forward kernel");
    return check_status(net);
}

static lb_status run_grad(lb_mlp* net, long long n, const float* feat, const float* target) {
    LB_MCUDA(cudaMemsetAsync(net->g, 0, sizeof(float) * NPARAM, net->stream), "memset");
    LB_MCUDA(cudaMemsetAsync(net->sse, 0, sizeof(float), net->stream), "memset");
    const long long tiles = (n + tc::M - 1) / tc::M;
    const unsigned grid = (unsigned)std::max<long long>(1, std::min<long long>(tiles, 152LL));
    km_grad_tc<<<grid, tc::M, tc::GSMEM, net->stream>>>(net->p, n, feat, target, net->g, net->sse, net->status,
                                                       net->wait_polls);
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

static void adam_step(lb_mlp* net, float lr) {
    net->t += 1;
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = 1.0f - powf(b1, (float)net->t), c2 = 1.0f - powf(b2, (float)net->t);
    km_adam<<<(NPARAM + 255) / 256, 256, 0, net->stream>>>(net->p, net->g, net->m, net->v, lr, b1, b2, 1e-8f, c1, c2);
}

lb_status lb_mlp_train_step(lb_mlp* net, long long n, const float* feat, const float* target, float lr, float* sse) {
    if (!net || n < 1 || !feat || !target || !(lr > 0)) return mfail(net, LB_ERR_ARG, "lb_mlp_train_step: bad argument");
    lb_status s = run_grad(net, n, feat, target);
    if (s != LB_OK) return s;
    adam_step(net, lr);
    LB_MCUDA(cudaGetLastError(), "adam kernel");
    if (sse) LB_MCUDA(cudaMemcpyAsync(sse, net->sse, sizeof(float), cudaMemcpyDefault, net->stream), "copy");
    return LB_OK;
}

lb_status lb_mlp_train(lb_mlp* net, long long n, const float* feat, const float* target, float target_scale,
                       int batch, int steps, float lr, unsigned long long seed, int loss_every, float* loss) {
    if (!net || n < 1 || !feat || !target || batch < 1 || steps < 1 || !(lr > 0) || !(target_scale > 0) ||
        !isfinite(target_scale) || loss_every < 1)
        return mfail(net, LB_ERR_ARG, "lb_mlp_train: bad argument");
    const int nrec = (steps - 1) / loss_every + 2;
    const size_t need = (size_t)batch * (D0 + D3) + (size_t)nrec;
    if (need > net->mb_floats) {
        LB_MCUDA(cudaStreamSynchronize(net->stream), "stream synchronize");
        cudaFree(net->mb);
        net->mb = nullptr;
        net->mb_floats = 0;
        LB_MCUDA(cudaMalloc(&net->mb, sizeof(float) * need), "minibatch buffers");
        net->mb_floats = need;
    }
    float* bfeat = net->mb;
    float* btarget = bfeat + (size_t)batch * D0;
    float* rec = btarget + (size_t)batch * D3;
    const float inv_count = 1.0f / (3.0f * (float)batch);
    int k = 0;
    for (int s = 0; s < steps; ++s) {
        km_gather<<<(batch + 127) / 128, 128, 0, net->stream>>>(seed, s, batch, n, feat, target, 1.0f / target_scale,
                                                                bfeat, btarget);
        LB_MCUDA(cudaGetLastError(), "minibatch kernel");
        lb_status st = run_grad(net, batch, bfeat, btarget);
        if (st != LB_OK) return st;
        if (s % loss_every == 0 || s == steps - 1) km_record_loss<<<1, 1, 0, net->stream>>>(net->sse, inv_count, rec, k++);
        const float lr_s = fmaxf(lr * 0.5f * (1.0f + cosf(3.14159265358979f * (float)s / (float)steps)), 1e-6f);
        adam_step(net, lr_s);
        LB_MCUDA(cudaGetLastError(), "adam kernel");
    }
    if (loss) LB_MCUDA(cudaMemcpyAsync(loss, rec, sizeof(float) * k, cudaMemcpyDefault, net->stream), "loss copy");
    LB_MCUDA(cudaStreamSynchronize(net->stream), "stream synchronize");
    return LB_OK;
}

}  // extern "C"
