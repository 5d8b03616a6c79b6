// Learned surrogate of the single-scatter sum: a 4-layer MLP
//   x (32, BF16) -> 128 -> 128 -> 128 (GELU, tanh form) -> 1
// predicting ln(S_w + eps) for one (event, voxel, line), where S_w is the
// single-scatter part of the system-matrix element for line w (Eq. s_p with
// n = 1 summed over the scatter points).  Two families of kernels, all
// written here, BF16 operands with FP32 accumulation:
//  * inference (k_tc_forward and the row kernel k_surrogate_rows) and the
//    training forward (k_tc_forward with stored pre-activations): tcgen05
//    MMAs from swizzled shared memory into tensor memory, described below;
//  * training backward (k_tc_back_layer per hidden layer, tcgen05; the
//    output layer k_back_out and the Adam update on the CUDA cores).
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstring>
#include <vector>

#include "lmmew_internal.cuh"

namespace lmmew {
namespace mlp {

constexpr int kIn = 32, kHid = 128;
constexpr int kTile = 128;       // samples per CTA
constexpr int kThreads = 256;
// parameter vector (FP32 masters): W1[128][32] b1 W2[128][128] b2 W3 b3 w4[128] b4
constexpr int kOffW1 = 0, kOffB1 = kOffW1 + kHid * kIn, kOffW2 = kOffB1 + kHid,
              kOffB2 = kOffW2 + kHid * kHid, kOffW3 = kOffB2 + kHid,
              kOffB3 = kOffW3 + kHid * kHid, kOffW4 = kOffB3 + kHid, kOffB4 = kOffW4 + kHid,
              kParams = kOffB4 + 1;

typedef __nv_bfloat16 bf16;

// GELU, tanh form: 0.5 z (1 + tanh(u)), u = sqrt(2/pi) (z + 0.044715 z^3),
// evaluated as u = z (c + c k z^2), h = hz tanh(u) + hz with hz = z / 2.  The
// packed doubled form below performs the same IEEE operations scaled by the
// exact factor 2, so every kernel produces the same activations.
constexpr float kGeluC = 0.7978845608028654f;
constexpr float kGeluCK = 0.7978845608028654f * 0.044715f;
__device__ __forceinline__ float tanh_fast(float x) {
    float y;
    asm("tanh.approx.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float gelu(float z) {
    const float u = z * fmaf(z * z, kGeluCK, kGeluC);
    const float hz = z * 0.5f;
    return fmaf(hz, tanh_fast(u), hz);
}
// 2 gelu(z) = z + z tanh(u): the tensor-core kernels fold the factor 1/2 into
// the next layer's weights (an exact power-of-two scaling, so the BF16
// activations and every product come out bit for bit the same).
__device__ __forceinline__ f32x2 gelu2_doubled(f32x2 z) {
    const f32x2 u = mul2(z, fma2(mul2(z, z), pk(kGeluCK, kGeluCK), pk(kGeluC, kGeluC)));
    float u0, u1;
    upk(u, u0, u1);
    return fma2(z, pk(tanh_fast(u0), tanh_fast(u1)), z);
}
__device__ __forceinline__ float gelu_grad(float z) {
    const float u = 0.7978845608028654f * (z + 0.044715f * z * z * z);
    const float t = tanh_fast(u);
    return 0.5f * (1.f + t) +
           0.5f * z * (1.f - t * t) * 0.7978845608028654f * (1.f + 3.f * 0.044715f * z * z);
}

struct Weights {
    const bf16* W1;    // [128][32]
    const bf16* W2;    // [128][128]
    const bf16* W3;
    const float* p;    // FP32 parameters (biases, w4, b4)
};

// Output layer backward.  loss = (1/n) sum_i v_i (out_i - t_i)^2 with sample
// weights v_i (1 when weight is null).  dZ3 = dout w4 gelu'(Z3); per-CTA
// partial sums of dL/dw4 and dL/db4.
__global__ void __launch_bounds__(kThreads) k_back_out(const float* p, const float* out,
                                                       const float* target, const float* weight,
                                                       const bf16* z3, int64_t n, float inv_n,
                                                       bf16* dz3, float* part /* [cta][kHid + 1] */) {
    __shared__ float dout[kTile];
    const int64_t base = (int64_t)blockIdx.x * kTile;
    const int rows = (n - base) < kTile ? (int)(n - base) : kTile;
    if (threadIdx.x < kTile) {
        float d = 0.f;
        if (threadIdx.x < rows) {
            const int64_t i = base + threadIdx.x;
            d = 2.f * inv_n * (out[i] - target[i]);
            if (weight) d *= weight[i];
        }
        dout[threadIdx.x] = d;
    }
    __syncthreads();
    // each thread keeps one column c; its partial of dL/dw4[c] over the rows
    // it visits is combined with the other thread of that column at the end
    __shared__ float colsum[kThreads];
    float s = 0.f;
    const int c = threadIdx.x % kHid;
    const float w4c = p[kOffW4 + c];
    constexpr int kRowsPerThread = kTile * kHid / kThreads;   // rows r0 + 2 k
    constexpr int kBatch = 8;                                  // loads in flight together
    for (int k0 = 0; k0 < kRowsPerThread; k0 += kBatch) {
        float z[kBatch];
#pragma unroll
        for (int k = 0; k < kBatch; ++k) {
            const int r = (threadIdx.x + (k0 + k) * kThreads) / kHid;
            z[k] = r < rows ? __bfloat162float(z3[(size_t)(base + r) * kHid + c]) : 0.f;
        }
#pragma unroll
        for (int k = 0; k < kBatch; ++k) {
            const int r = (threadIdx.x + (k0 + k) * kThreads) / kHid;
            float v = 0.f;
            if (r < rows) {
                v = dout[r] * w4c * gelu_grad(z[k]);
                s += dout[r] * gelu(z[k]);
            }
            dz3[(size_t)(base + r) * kHid + c] = __float2bfloat16_rn(v);
        }
    }
    colsum[threadIdx.x] = s;
    __syncthreads();
    static_assert(kThreads % kHid == 0, "whole columns per thread");
    if (threadIdx.x < kHid) {
        float tot = 0.f;
        for (int k = threadIdx.x; k < kThreads; k += kHid) tot += colsum[k];
        part[(size_t)blockIdx.x * (kHid + 1) + threadIdx.x] = tot;
    }
    if (threadIdx.x == kHid) {
        float sb = 0.f;
        for (int r = 0; r < rows; ++r) sb += dout[r];
        part[(size_t)blockIdx.x * (kHid + 1) + kHid] = sb;
    }
}

// Sum the per-CTA partials in CTA order into the gradient vector.
__global__ void k_reduce_grad(const float* pw1, const float* pb1, const float* pw2,
                              const float* pb2, const float* pw3, const float* pb3,
                              const float* pout, int n_cta, float* grad) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= kParams) return;
    const float* src;
    int stride, off;
    if (i < kOffB1) { src = pw1; stride = kHid * kIn; off = i - kOffW1; }
    else if (i < kOffW2) { src = pb1; stride = kHid; off = i - kOffB1; }
    else if (i < kOffB2) { src = pw2; stride = kHid * kHid; off = i - kOffW2; }
    else if (i < kOffW3) { src = pb2; stride = kHid; off = i - kOffB2; }
    else if (i < kOffB3) { src = pw3; stride = kHid * kHid; off = i - kOffW3; }
    else if (i < kOffW4) { src = pb3; stride = kHid; off = i - kOffB3; }
    else { src = pout; stride = kHid + 1; off = i - kOffW4; }
    float s = 0.f;
    for (int c = 0; c < n_cta; ++c) s += src[(size_t)c * stride + off];
    grad[i] = s;
}

__global__ void k_adam(float* p, float* m1, float* m2, const float* grad, float lr, float b1,
                       float b2, float eps, float c1, float c2, bf16* W1, bf16* W2, bf16* W3) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= kParams) return;
    const float gi = grad[i];
    const float a = b1 * m1[i] + (1.f - b1) * gi;
    const float v = b2 * m2[i] + (1.f - b2) * gi * gi;
    m1[i] = a;
    m2[i] = v;
    const float np = p[i] - lr * (a / c1) / (sqrtf(v / c2) + eps);
    p[i] = np;
    if (i < kOffB1) W1[i - kOffW1] = __float2bfloat16_rn(np);
    else if (i >= kOffW2 && i < kOffB2) W2[i - kOffW2] = __float2bfloat16_rn(np);
    else if (i >= kOffW3 && i < kOffB3) W3[i - kOffW3] = __float2bfloat16_rn(np);
}

__global__ void k_to_bf16(const float* src, int64_t n, bf16* dst) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) dst[i] = __float2bfloat16_rn(src[i]);
}

__global__ void k_mse(const float* out, const float* target, const float* weight, int64_t n,
                      double* acc) {
    __shared__ double red[256];
    double s = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * 256 + threadIdx.x; i < n; i += (int64_t)gridDim.x * 256) {
        const double d = (double)out[i] - target[i];
        s += (weight ? (double)weight[i] : 1.0) * d * d;
    }
    red[threadIdx.x] = s;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) acc[blockIdx.x] = red[0];
}

// batch gather for SGD: idx[i] -> rows of x (BF16), targets and weights
__global__ void k_gather_batch_rows(const bf16* x, const float* t, const float* v,
                                    const uint32_t* idx, int n, bf16* xb, float* tb, float* vb) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n * (kIn / 8)) return;
    const int r = i / (kIn / 8), c = (i % (kIn / 8)) * 8;
    const uint32_t s = idx[r];
    *reinterpret_cast<uint4*>(xb + (size_t)r * kIn + c) =
        *reinterpret_cast<const uint4*>(x + (size_t)s * kIn + c);
    if (c == 0) {
        tb[r] = t[s];
        if (v) vb[r] = v[s];
    }
}

// Sample weights of the training set: v_i = exp(gamma (t_i - max t)),
// normalised to mean 1.  One CTA of 1024 threads: max, then the weights and
// their sum, then the scaling.
__global__ void __launch_bounds__(1024) k_train_weights(const float* t, int64_t n, float gamma,
                                                        float* v) {
    __shared__ float redf[1024];
    __shared__ double redd[1024];
    float mx = -3.0e38f;
    for (int64_t i = threadIdx.x; i < n; i += 1024) mx = fmaxf(mx, t[i]);
    redf[threadIdx.x] = mx;
    __syncthreads();
    for (int o = 512; o > 0; o >>= 1) {
        if (threadIdx.x < o) redf[threadIdx.x] = fmaxf(redf[threadIdx.x], redf[threadIdx.x + o]);
        __syncthreads();
    }
    const float tmax = redf[0];
    double sum = 0.0;
    for (int64_t i = threadIdx.x; i < n; i += 1024) {
        const float w = __expf(gamma * (t[i] - tmax));
        v[i] = w;
        sum += w;
    }
    redd[threadIdx.x] = sum;
    __syncthreads();
    for (int o = 512; o > 0; o >>= 1) {
        if (threadIdx.x < o) redd[threadIdx.x] += redd[threadIdx.x + o];
        __syncthreads();
    }
    const float scale = (float)((double)n / redd[0]);
    for (int64_t i = threadIdx.x; i < n; i += 1024) v[i] *= scale;
}

// counter-based random index (SplitMix64 of (seed, step, i))
__device__ __forceinline__ uint64_t splitmix(uint64_t z) {
    z += 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}
__global__ void k_batch_indices(uint64_t seed, uint64_t step, int n, uint64_t n_total,
                                uint32_t* idx) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) idx[i] = (uint32_t)(splitmix(seed ^ splitmix(step * 0x100000001b3ull + i)) % n_total);
}


// ---------------------------------------------------------------------------
// Tensor-core (tcgen05) forward pass of the network, for inference.
//
// One CTA of 512 threads per SM, split into four independent groups of 128
// threads (one warp per 32-lane quarter of tensor memory) that share the
// weights: W1 (K padded from 32 to 64), W2 and W3 stay in shared memory in the
// canonical K-major layout with 128-byte swizzle (8-row x 128-byte atoms,
// 16-byte chunk j of row r stored at chunk j ^ (r mod 8), 64-element K blocks
// one after the other).  Each group owns a hidden tile H (128 samples x 128)
// in the same layout -- its first K block doubles as the input tile X, which
// the layer-0 MMAs have consumed before the first epilogue overwrites it --
// 128 columns of tensor memory, an mbarrier and a named barrier, and works
// through its own tiles of 128 samples: per layer one of its threads issues
// the M = 128 x N = 128 x K = 16 MMAs (kind::f16, BF16 operands, FP32
// accumulator) and commits them to the group's mbarrier; each warp then reads
// its 32 TMEM lanes (its samples) x 128 columns with tcgen05.ld, adds the
// bias, applies GELU and writes BF16 into H (the next layer's A operand) --
// or, after the last layer, the dot with the output weights.  While some
// groups wait for their MMAs the others compute, so the tensor core and the
// epilogues overlap.
constexpr int kTcThreads = 512;
constexpr int kTcGroups = 4;
constexpr int kGrpThreads = 128;
constexpr uint32_t kTcCols = 512;                  // TMEM columns: 128 per group (FP32 128 x 128)
constexpr uint32_t kAtomBlock = 128 * 128;         // bytes of one 64-wide K block of a 128-row tile
constexpr uint32_t kTcOffW1 = 0;                   // 128 x 64
constexpr uint32_t kTcOffW2 = kTcOffW1 + kAtomBlock;       // 128 x 128
constexpr uint32_t kTcOffW3 = kTcOffW2 + 2 * kAtomBlock;   // 128 x 128
constexpr uint32_t kTcOffG = kTcOffW3 + 2 * kAtomBlock;    // group tiles H (X = its first block)
constexpr uint32_t kGrpTiles = 2 * kAtomBlock;
constexpr uint32_t kTcOffF = kTcOffG + kTcGroups * kGrpTiles;   // floats: bias [3][128], w4 [128]
constexpr uint32_t kTcOffGF = kTcOffF + 4 * 128 * 4;            // per group: unit data
// unit data per group: voxel centres, voxel line integrals, event (energy,
// bin centre); then, for the surrogate rows, per line the number of events
// its single scatter can reach, per-warp counts and the events' indices
constexpr uint32_t kGrpUnitFloats = 32 * 2 + 32 * 8 + 128 * 2;
constexpr uint32_t kGrpFloats =
    kGrpUnitFloats + LMMEW_MAX_LINES + 4 * LMMEW_MAX_LINES + LMMEW_MAX_LINES * 128 / 4;
constexpr uint32_t kTcOffBar = kTcOffGF + kTcGroups * kGrpFloats * 4;   // mbarriers, TMEM, abort
constexpr size_t kTcSmem = kTcOffBar + 64 + 1024;          // + room to align the base to 1 KB
static_assert(kTcOffW2 % 1024 == 0 && kTcOffW3 % 1024 == 0 && kTcOffG % 1024 == 0 &&
                  kGrpTiles % 1024 == 0, "swizzle atoms need 1 KB alignment");
static_assert(kTcSmem <= 227 * 1024, "shared memory");
// instruction descriptor: FP32 accumulator, BF16 A and B, both K-major, N = 128, M = 128
constexpr uint32_t kTcIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((128u >> 3) << 17) |
                              ((128u >> 4) << 24);

// Byte offset of 16-byte chunk j (0..7) of K block kb of row r in a 128-row tile.
__device__ __forceinline__ uint32_t sw_chunk(int r, int kb, int j) {
    return (uint32_t)kb * kAtomBlock + (uint32_t)r * 128u + ((uint32_t)(j ^ (r & 7)) << 4);
}
// Shared-memory matrix descriptor of a K-major, 128-byte-swizzled operand
// starting at byte address saddr (8-row groups 1024 bytes apart).
__device__ __forceinline__ uint64_t umma_desc(uint32_t saddr) {
    uint64_t d = (uint64_t)((saddr & 0x3FFFFu) >> 4);
    d |= (uint64_t)1 << 16;             // leading byte offset (unused within a swizzle atom)
    d |= (uint64_t)(1024 >> 4) << 32;   // stride byte offset
    d |= (uint64_t)1 << 46;             // descriptor version
    d |= (uint64_t)2 << 61;             // 128-byte swizzle
    return d;
}
__device__ __forceinline__ void tc_alloc(uint32_t slot, uint32_t ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(slot),
                 "r"(ncols) : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tc_dealloc(uint32_t taddr, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols)
                 : "memory");
}
__device__ __forceinline__ void tc_mma(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc,
                                       uint32_t accumulate) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(d),
        "l"(a), "l"(b), "r"(idesc), "r"(accumulate)
        : "memory");
}
__device__ __forceinline__ void tc_commit(uint32_t bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
                 : "memory");
}
__device__ __forceinline__ void tc_fence_before() {
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void fence_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
// 32 consecutive FP32 columns of this thread's TMEM lane.
__device__ __forceinline__ void tc_ld32(uint32_t taddr, float* v) {
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, "
        "%12, %13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, "
        "%30, %31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
          "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]),
          "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]),
          "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr)
        : "memory");
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

// 16 consecutive FP32 columns of this thread's TMEM lane, left in flight:
// the registers hold the values only after tc_wait_ld16 on the same array,
// whose asm names them as written (so no use is moved above the wait).
__device__ __forceinline__ void tc_ld16_start(uint32_t taddr, uint32_t (&r)[16]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, "
        "%11, %12, %13, %14, %15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
          "=r"(r[14]), "=r"(r[15])
        : "r"(taddr)
        : "memory");
}
__device__ __forceinline__ void tc_wait_ld16(uint32_t (&r)[16]) {
    asm volatile("tcgen05.wait::ld.sync.aligned;"
                 : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]),
                   "+r"(r[6]), "+r"(r[7]), "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11]),
                   "+r"(r[12]), "+r"(r[13]), "+r"(r[14]), "+r"(r[15])
                 :
                 : "memory");
}

struct TcShared {
    unsigned char* base;   // 1 KB aligned
    uint32_t sbase;        // its shared-window address
    uint32_t* tmem_slot;
    int* abort;            // [4]: set by a group's issuing thread when its MMA wait ran out
};

__device__ __forceinline__ TcShared tc_shared(unsigned char* raw) {
    TcShared t;
    const uint32_t a = (uint32_t)__cvta_generic_to_shared(raw);
    const uint32_t pad = ((a + 1023u) & ~1023u) - a;
    t.base = raw + pad;
    t.sbase = a + pad;
    t.tmem_slot = reinterpret_cast<uint32_t*>(t.base + kTcOffBar + 32);
    t.abort = reinterpret_cast<int*>(t.base + kTcOffBar + 40);
    return t;
}

// One of the four thread groups of the CTA and its private resources.
struct TcGroup {
    int g;          // 0..3
    int gt;         // thread index in the group, 0..127 (= the sample row it owns)
    uint32_t h;     // byte offset of the group's hidden tile; X is its first K block
    float* f;       // the group's unit data
    uint32_t tmem;  // its 128 accumulator columns
    uint32_t bar;   // its mbarrier
};

__device__ __forceinline__ TcGroup tc_group(const TcShared& S, uint32_t tmem_base) {
    TcGroup G;
    G.g = threadIdx.x >> 7;
    G.gt = threadIdx.x & 127;
    G.h = kTcOffG + (uint32_t)G.g * kGrpTiles;
    G.f = reinterpret_cast<float*>(S.base + kTcOffGF) + G.g * kGrpFloats;
    G.tmem = tmem_base + (uint32_t)G.g * 128u;
    G.bar = S.sbase + kTcOffBar + 8u * (uint32_t)G.g;
    return G;
}

__device__ __forceinline__ void group_sync(int g) {
    asm volatile("bar.sync %0, 128;" ::"r"(g + 1) : "memory");
}

// Weights into their swizzled tiles, the mbarriers initialised, TMEM
// allocated (warp 0).  Ends with a CTA barrier; returns the TMEM base address.
__device__ uint32_t tc_setup(const TcShared& S, const Weights& w) {
    const int tid = threadIdx.x;
    // W1 with b1 in input columns 32 (BF16 high part) and 33 (the remainder), so
    // the first layer's bias comes out of the MMA (the inputs carry 1 there)
    for (int i = tid; i < 128 * 8; i += kTcThreads) {
        const int n = i >> 3, j = i & 7;
        uint4 v = make_uint4(0u, 0u, 0u, 0u);
        if (j < 4) {
            v = *reinterpret_cast<const uint4*>(w.W1 + (size_t)n * kIn + j * 8);
        } else if (j == 4) {
            const float b = w.p[kOffB1 + n];
            const __nv_bfloat16 hi = __float2bfloat16_rn(b);
            const __nv_bfloat162 t = __halves2bfloat162(hi, __float2bfloat16_rn(b - __bfloat162float(hi)));
            v.x = *reinterpret_cast<const uint32_t*>(&t);
        }
        *reinterpret_cast<uint4*>(S.base + kTcOffW1 + sw_chunk(n, 0, j)) = v;
    }
    // W2, W3 halved: the activations feeding them are 2 gelu
    const __nv_bfloat162 half2 = __float2bfloat162_rn(0.5f);
    for (int i = tid; i < 128 * 16; i += kTcThreads) {
        const int n = i >> 4, c = i & 15;
        uint4 a = *reinterpret_cast<const uint4*>(w.W2 + (size_t)n * kHid + c * 8);
        uint4 b = *reinterpret_cast<const uint4*>(w.W3 + (size_t)n * kHid + c * 8);
        __nv_bfloat162* pa = reinterpret_cast<__nv_bfloat162*>(&a);
        __nv_bfloat162* pb = reinterpret_cast<__nv_bfloat162*>(&b);
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            pa[k] = __hmul2(pa[k], half2);
            pb[k] = __hmul2(pb[k], half2);
        }
        *reinterpret_cast<uint4*>(S.base + kTcOffW2 + sw_chunk(n, c >> 3, c & 7)) = a;
        *reinterpret_cast<uint4*>(S.base + kTcOffW3 + sw_chunk(n, c >> 3, c & 7)) = b;
    }
    float* F = reinterpret_cast<float*>(S.base + kTcOffF);
    for (int i = tid; i < 3 * kHid; i += kTcThreads) {
        const int l = i / kHid;
        F[i] = l == 0 ? 0.f : w.p[(l == 1 ? kOffB2 : kOffB3) + i % kHid];
    }
    for (int i = tid; i < kHid; i += kTcThreads) F[3 * kHid + i] = 0.5f * w.p[kOffW4 + i];
    if (tid == 0) {
        for (int g = 0; g < kTcGroups; ++g) {
            mbar_init(S.sbase + kTcOffBar + 8 * g, 1);
            S.abort[g] = 0;
        }
        mbar_fence_init();
    }
    if (tid < 32) tc_alloc(S.sbase + kTcOffBar + 32, kTcCols);
    fence_async_smem();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    return *S.tmem_slot;
}

// After an MMA wait ran out, each group waits once more (bounded) for its MMAs
// in flight before the tensor memory they write is released.
__device__ void tc_teardown(const TcShared& S, const TcGroup& G, uint32_t tmem_base,
                            uint32_t phase) {
    tc_fence_before();
    __syncthreads();
    if (G.gt == 0 && S.abort[G.g] && phase > 0) mbar_wait_bounded(G.bar, (phase - 1) & 1);
    __syncthreads();
    tc_fence_after();
    if (threadIdx.x < 32) tc_dealloc(tmem_base, kTcCols);
}

// Input chunks 4..7 of every row of the group's X: columns 32, 33 carry 1
// (the first layer's bias), 34..63 zero.  Written with the inputs each pass,
// since the hidden layers overwrite X.
__device__ __forceinline__ void tc_input_constants(const TcShared& S, const TcGroup& G) {
    const __nv_bfloat162 one2 = __float2bfloat162_rn(1.f);
    for (int k = G.gt; k < 128 * 4; k += kGrpThreads) {
        const int r = k & 127, j = 4 + (k >> 7);
        uint4 v = make_uint4(0u, 0u, 0u, 0u);
        if (j == 4) v.x = *reinterpret_cast<const uint32_t*>(&one2);
        *reinterpret_cast<uint4*>(S.base + G.h + sw_chunk(r, 0, j)) = v;
    }
}

// The network on the group's 128 samples whose inputs sit in X (written,
// fenced and followed by a group barrier).  Returns in every thread the output
// of sample (group thread index); false if an MMA wait ran out (the status
// word is set and the caller stops).  With kStoreZ (training) the thread also
// stores its sample's pre-activations of the three hidden layers, BF16, at
// z_row + layer * z_stride (z_row null: a padding sample, nothing stored).
// The last layer ends without a group barrier: a warp goes on to its next
// samples' inputs while the others finish, and the barrier the caller
// places after writing the next inputs also orders every warp's last TMEM
// loads before the next MMAs.  A wait that ran out in the last layer is
// therefore seen by the whole group at the next call's entry (after that
// barrier), so every thread of the group stops at the same point.
template <bool kStoreZ>
__device__ bool tc_network(const TcShared& S, const TcGroup& G, uint32_t& phase, float b4,
                           float* out_row, int* status, bf16* z_row = nullptr,
                           size_t z_stride = 0) {
    if (S.abort[G.g]) return false;
    const int lq = G.gt >> 5;
    const int row = G.gt;
    const float* F = reinterpret_cast<const float*>(S.base + kTcOffF);
    f32x2 sacc2 = pk(0.f, 0.f);   // output layer: even and odd columns
    // descriptors of the operands' first K slices; a slice off bytes further
    // on is the same descriptor plus off / 16 (the 14-bit address field of a
    // shared-memory operand below 256 KB does not carry)
    const uint64_t da = umma_desc(S.sbase + G.h);
    // the three layers one after the other, each specialised at compile time
#pragma unroll
    for (int layer = 0; layer < 3; ++layer) {
        if (G.gt == 0) {
            tc_fence_after();
            const uint64_t db =
                umma_desc(S.sbase + (layer == 0 ? kTcOffW1 : layer == 1 ? kTcOffW2 : kTcOffW3));
            constexpr int kMaxSteps = 8;
#pragma unroll
            for (int ks = 0; ks < kMaxSteps; ++ks) {
                if (layer == 0 && ks >= 4) break;
                const uint32_t off = (uint32_t)(ks >> 2) * kAtomBlock + (uint32_t)(ks & 3) * 32u;
                tc_mma(G.tmem, da + (off >> 4), db + (off >> 4), kTcIdesc, ks > 0 ? 1u : 0u);
            }
            tc_commit(G.bar);
        }
        // every thread waits for the MMAs itself (no group barrier here); a
        // warp in which a wait ran out skips the epilogue (its TMEM loads are
        // warp-collective) and flags the group, which stops after the barrier
        // that ends the layer
        const bool done = __all_sync(0xffffffffu, mbar_wait_bounded(G.bar, phase & 1));
        ++phase;
        if (!done) {
            S.abort[G.g] = 1;
            atomicOr(status, kStatusTimeout);
        }
        tc_fence_after();
        if (done) {
            // 16-column chunks; the next chunk's TMEM load is in flight while
            // this one is computed (same operations, in the same column
            // order, as one chunk at a time)
            const uint32_t tlane = G.tmem + ((uint32_t)(lq * 32) << 16);
            auto chunk = [&](int cc, uint32_t(&v)[16]) {
                const int cb = cc * 16;   // columns cb .. cb + 15
                const float4* bias4 = reinterpret_cast<const float4*>(F + layer * kHid + cb);
                if (layer < 2) {
                    uint32_t hb[8];
#pragma unroll
                    for (int i = 0; i < 16; i += 4) {
                        f32x2 z0 = pk(__uint_as_float(v[i]), __uint_as_float(v[i + 1]));
                        f32x2 z1 = pk(__uint_as_float(v[i + 2]), __uint_as_float(v[i + 3]));
                        if (layer > 0) {   // the first layer's bias comes out of the MMA
                            const float4 b = bias4[i >> 2];
                            z0 = add2(z0, pk(b.x, b.y));
                            z1 = add2(z1, pk(b.z, b.w));
                        }
                        if (kStoreZ && z_row) {
                            float a0, a1, a2, a3;
                            upk(z0, a0, a1);
                            upk(z1, a2, a3);
                            __nv_bfloat162* zp = reinterpret_cast<__nv_bfloat162*>(
                                z_row + layer * z_stride + cb + i);
                            zp[0] = __floats2bfloat162_rn(a0, a1);
                            zp[1] = __floats2bfloat162_rn(a2, a3);
                        }
                        float h0, h1, h2, h3;
                        upk(gelu2_doubled(z0), h0, h1);
                        upk(gelu2_doubled(z1), h2, h3);
                        const __nv_bfloat162 t0 = __floats2bfloat162_rn(h0, h1);
                        const __nv_bfloat162 t1 = __floats2bfloat162_rn(h2, h3);
                        hb[i >> 1] = *reinterpret_cast<const uint32_t*>(&t0);
                        hb[(i >> 1) + 1] = *reinterpret_cast<const uint32_t*>(&t1);
                    }
                    // 16 columns: two 16-byte chunks of K block cc / 4
#pragma unroll
                    for (int c = 0; c < 2; ++c)
                        *reinterpret_cast<uint4*>(S.base + G.h + sw_chunk(row, cc >> 2, (cc & 3) * 2 + c)) =
                            make_uint4(hb[4 * c], hb[4 * c + 1], hb[4 * c + 2], hb[4 * c + 3]);
                } else {
                    const float4* w44 = reinterpret_cast<const float4*>(F + 3 * kHid + cb);
#pragma unroll
                    for (int i = 0; i < 16; i += 4) {
                        const float4 b = bias4[i >> 2], ww = w44[i >> 2];
                        const f32x2 z0 = add2(pk(__uint_as_float(v[i]), __uint_as_float(v[i + 1])),
                                              pk(b.x, b.y));
                        const f32x2 z1 = add2(pk(__uint_as_float(v[i + 2]), __uint_as_float(v[i + 3])),
                                              pk(b.z, b.w));
                        if (kStoreZ && z_row) {
                            float a0, a1, a2, a3;
                            upk(z0, a0, a1);
                            upk(z1, a2, a3);
                            __nv_bfloat162* zp = reinterpret_cast<__nv_bfloat162*>(
                                z_row + layer * z_stride + cb + i);
                            zp[0] = __floats2bfloat162_rn(a0, a1);
                            zp[1] = __floats2bfloat162_rn(a2, a3);
                        }
                        sacc2 = fma2(gelu2_doubled(z0), pk(ww.x, ww.y), sacc2);
                        sacc2 = fma2(gelu2_doubled(z1), pk(ww.z, ww.w), sacc2);
                    }
                }
            };
            uint32_t ra[16], rb[16];
            tc_ld16_start(tlane, ra);
            tc_wait_ld16(ra);
#pragma unroll 1
            for (int cp = 0; cp < 8; cp += 2) {   // pairs of chunks: ra, then rb
                tc_ld16_start(tlane + (uint32_t)(cp + 1) * 16u, rb);
                chunk(cp, ra);
                tc_wait_ld16(rb);
                if (cp + 2 < 8) tc_ld16_start(tlane + (uint32_t)(cp + 2) * 16u, ra);
                chunk(cp + 1, rb);
                if (cp + 2 < 8) tc_wait_ld16(ra);
            }
        }
        tc_fence_before();
        if (layer < 2) {
            fence_async_smem();
            group_sync(G.g);
            if (S.abort[G.g]) return false;
        }
    }
    float s_even, s_odd;
    upk(sacc2, s_even, s_odd);
    *out_row = (s_even + s_odd) + b4;
    return true;
}

// Network outputs for n BF16 input rows; with kTrain also the pre-activations
// of the three hidden layers, BF16 [3][n][128] at z (the training forward).
template <bool kTrain>
__global__ void __launch_bounds__(kTcThreads, 1) k_tc_forward(Weights w, const bf16* x, int64_t n,
                                                              float* out, int* status,
                                                              bf16* z = nullptr) {
    extern __shared__ unsigned char smem_raw[];
    const TcShared S = tc_shared(smem_raw);
    const uint32_t tmem_base = tc_setup(S, w);
    const TcGroup G = tc_group(S, tmem_base);
    const float b4 = w.p[kOffB4];
    uint32_t phase = 0;
    const int64_t n_tiles = (n + 127) / 128;
    // tiles group-major across the CTAs, so that few tiles still use many SMs
    for (int64_t t = (int64_t)G.g * gridDim.x + blockIdx.x; t < n_tiles;
         t += (int64_t)gridDim.x * kTcGroups) {
        const int64_t base = t * 128;
        for (int k = G.gt; k < 128 * 4; k += kGrpThreads) {   // 128 rows x 4 chunks of 8 inputs
            const int r = k & 127, j = k >> 7;
            uint4 v = make_uint4(0u, 0u, 0u, 0u);
            if (base + r < n) v = *reinterpret_cast<const uint4*>(x + (size_t)(base + r) * kIn + j * 8);
            *reinterpret_cast<uint4*>(S.base + G.h + sw_chunk(r, 0, j)) = v;
        }
        tc_input_constants(S, G);
        fence_async_smem();
        group_sync(G.g);
        float o = 0.f;
        bf16* z_row = (kTrain && base + G.gt < n) ? z + (size_t)(base + G.gt) * kHid : nullptr;
        if (!tc_network<kTrain>(S, G, phase, b4, &o, status, z_row, (size_t)n * kHid)) break;
        if (base + G.gt < n) out[base + G.gt] = o;
    }
    tc_teardown(S, G, tmem_base, phase);
}

// ---------------------------------------------------------------------------
// Training backward on the tensor cores.  One hidden layer l with input
// width K (32 for the first layer, 128 otherwise); one CTA of 128 threads per
// tile of 128 samples:
//   gW[i][j] = sum_s dZ[s][i] H[s][j]        M = 128 outputs, N = K, K-dim = samples
//   dZprev[s][j] = (sum_i dZ[s][i] W[i][j]) gelu'(Zprev[s][j])      (l > 1)
//                                            M = 128 samples, N = 128, K-dim = outputs
// H = gelu(Zprev) for l > 1, the input x for l = 1.  Every operand is staged
// K-major in 128-byte-swizzled shared memory; the transposes (W^T, dZ^T,
// H^T) happen while staging from global memory.  Each CTA writes its partial
// sums of gW and of the bias gradient; k_reduce_grad adds them in CTA order.
constexpr uint32_t kBkBlock = 128 * 128;   // bytes of one 64-wide K block of a 128-row operand
template <int K>
struct BackTc {
    static constexpr uint32_t kADx = 0;                  // dZ   [128 samples][128 outputs]
    static constexpr uint32_t kBDx = 2 * kBkBlock;       // W^T  [128 inputs][128 outputs]
    static constexpr uint32_t kADw = 4 * kBkBlock;       // dZ^T [128 outputs][128 samples]
    static constexpr uint32_t kBDw = 6 * kBkBlock;       // H^T  [K inputs][128 samples]
    static constexpr uint32_t kBDwBlock = (uint32_t)K * 128u;
    static constexpr uint32_t kBar = kBDw + 2 * kBDwBlock;
    static constexpr size_t kSmem = kBar + 64 + 1024;     // + room to align the base to 1 KB
    static constexpr uint32_t kIdescDx = (1u << 4) | (1u << 7) | (1u << 10) |
                                         ((128u >> 3) << 17) | ((128u >> 4) << 24);
    static constexpr uint32_t kIdescDw = (1u << 4) | (1u << 7) | (1u << 10) |
                                         (((uint32_t)K >> 3) << 17) | ((128u >> 4) << 24);
    static_assert(K % 32 == 0 && K >= 32 && K <= 128, "N of the weight-gradient MMA");
    static_assert(kBDwBlock % 1024 == 0 && kSmem <= 227 * 1024, "shared memory");
};

// Byte offset of 16-byte chunk j (0..7) of K block kb of row r, blocks of
// `block` bytes (rows x 128 B).
__device__ __forceinline__ uint32_t sw_off(int r, int kb, int j, uint32_t block) {
    return (uint32_t)kb * block + (uint32_t)r * 128u + ((uint32_t)(j ^ (r & 7)) << 4);
}

__device__ __forceinline__ uint32_t bf16_pair(float lo, float hi) {
    const __nv_bfloat162 t = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<const uint32_t*>(&t);
}

template <int K>
__global__ void __launch_bounds__(128) k_tc_back_layer(const bf16* dz, const bf16* zprev,
                                                       const bf16* x, const bf16* W, int64_t n,
                                                       float* part_w /* [cta][128][K] */,
                                                       float* part_b /* [cta][128] */,
                                                       bf16* dzprev, int* status) {
    typedef BackTc<K> L;
    extern __shared__ unsigned char smem_raw[];
    const uint32_t a0 = (uint32_t)__cvta_generic_to_shared(smem_raw);
    const uint32_t pad = ((a0 + 1023u) & ~1023u) - a0;
    unsigned char* sm = smem_raw + pad;
    const uint32_t sb = a0 + pad;
    const uint32_t bar = sb + L::kBar;
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(sm + L::kBar + 16);
    int* abort_flag = reinterpret_cast<int*>(sm + L::kBar + 24);
    const int t = threadIdx.x, warp = t >> 5;
    const int64_t base = (int64_t)blockIdx.x * 128;
    const int rows = (n - base) < 128 ? (int)(n - base) : 128;
    // the previous layer's dZ exists only above the first layer (K = 128)
    const bool want_dx = K == kHid && dzprev != nullptr;
    if (t == 0) {
        mbar_init(bar, 1);
        *abort_flag = 0;
        mbar_fence_init();
    }
    if (warp == 0) tc_alloc(sb + L::kBar + 16, 256);
    // Transposed operands are built from coalesced 16-byte row loads: 8
    // consecutive elements of one source row go to 8 rows of the tile, each
    // into its 2-byte slot of the sample (or output) column.
    auto put_t = [&](uint32_t region, uint32_t block, int row, int col, uint16_t v) {
        *reinterpret_cast<uint16_t*>(sm + region + sw_off(row, col >> 6, (col & 63) >> 3, block) +
                                     (col & 7) * 2) = v;
    };
    // Every staging loop first loads all of its 16-byte vectors (independent
    // loads in flight together), then stores them.
    if (K == kHid && want_dx) {
        // dZ rows, K-major over the outputs; dZ^T [output][sample] from the same rows
        uint4 v[16];
#pragma unroll
        for (int k = 0; k < 16; ++k) {
            const int i = t + k * 128, r = i >> 4, c = i & 15;
            v[k] = r < rows ? *reinterpret_cast<const uint4*>(dz + (size_t)(base + r) * kHid + c * 8)
                            : make_uint4(0u, 0u, 0u, 0u);
        }
#pragma unroll
        for (int k = 0; k < 16; ++k) {
            const int i = t + k * 128, r = i >> 4, c = i & 15;
            *reinterpret_cast<uint4*>(sm + L::kADx + sw_off(r, c >> 3, c & 7, kBkBlock)) = v[k];
        }
        // W^T [input j][output o] from the rows of W [output o][input j]
#pragma unroll
        for (int k = 0; k < 16; ++k) {
            const int i = t + k * 128, o = i / (K / 8), jc = i % (K / 8);
            v[k] = *reinterpret_cast<const uint4*>(W + (size_t)o * K + jc * 8);
        }
#pragma unroll
        for (int k = 0; k < 16; ++k) {
            const int i = t + k * 128, o = i / (K / 8), jc = i % (K / 8);
            const uint16_t* e = reinterpret_cast<const uint16_t*>(&v[k]);
#pragma unroll
            for (int q = 0; q < 8; ++q) put_t(L::kBDx, kBkBlock, jc * 8 + q, o, e[q]);
        }
    }
    {
        // dZ^T [output i][sample s] from the rows of dZ [sample s][output i]
        uint4 v[16];
#pragma unroll
        for (int k = 0; k < 16; ++k) {
            const int i = t + k * 128, r = i >> 4, c = i & 15;
            v[k] = r < rows ? *reinterpret_cast<const uint4*>(dz + (size_t)(base + r) * kHid + c * 8)
                            : make_uint4(0u, 0u, 0u, 0u);
        }
#pragma unroll
        for (int k = 0; k < 16; ++k) {
            const int i = t + k * 128, r = i >> 4, c = i & 15;
            const uint16_t* e = reinterpret_cast<const uint16_t*>(&v[k]);
#pragma unroll
            for (int q = 0; q < 8; ++q) put_t(L::kADw, kBkBlock, c * 8 + q, r, e[q]);
        }
    }
    {
        // H^T [input j][sample s]; H = gelu(Zprev) above the first layer, else x
        constexpr int kLoads = K / 8;   // 16-byte vectors per thread
        uint4 v[kLoads];
#pragma unroll
        for (int k = 0; k < kLoads; ++k) {
            const int i = t + k * 128, r = i / (K / 8), jc = i % (K / 8);
            v[k] = r >= rows ? make_uint4(0u, 0u, 0u, 0u)
                   : zprev   ? *reinterpret_cast<const uint4*>(zprev + (size_t)(base + r) * kHid + jc * 8)
                             : *reinterpret_cast<const uint4*>(x + (size_t)(base + r) * kIn + jc * 8);
        }
#pragma unroll
        for (int k = 0; k < kLoads; ++k) {
            const int i = t + k * 128, r = i / (K / 8), jc = i % (K / 8);
            const __nv_bfloat162* e = reinterpret_cast<const __nv_bfloat162*>(&v[k]);
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const float2 f = __bfloat1622float2(e[q]);
                // padding rows are zero, and gelu(0) = 0
                const __nv_bfloat16 b0 = __float2bfloat16_rn(zprev ? gelu(f.x) : f.x);
                const __nv_bfloat16 b1 = __float2bfloat16_rn(zprev ? gelu(f.y) : f.y);
                put_t(L::kBDw, L::kBDwBlock, jc * 8 + 2 * q, r, *reinterpret_cast<const uint16_t*>(&b0));
                put_t(L::kBDw, L::kBDwBlock, jc * 8 + 2 * q + 1, r, *reinterpret_cast<const uint16_t*>(&b1));
            }
        }
    }
    fence_async_smem();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;
    if (t == 0) {
        if (want_dx) {
            for (int ks = 0; ks < 8; ++ks) {
                const uint32_t off = (uint32_t)(ks >> 2) * kBkBlock + (uint32_t)(ks & 3) * 32u;
                tc_mma(tmem, umma_desc(sb + L::kADx + off), umma_desc(sb + L::kBDx + off),
                       L::kIdescDx, ks > 0 ? 1u : 0u);
            }
        }
        for (int ks = 0; ks < 8; ++ks) {
            const uint32_t oa = (uint32_t)(ks >> 2) * kBkBlock + (uint32_t)(ks & 3) * 32u;
            const uint32_t ob = (uint32_t)(ks >> 2) * L::kBDwBlock + (uint32_t)(ks & 3) * 32u;
            tc_mma(tmem + 128u, umma_desc(sb + L::kADw + oa), umma_desc(sb + L::kBDw + ob),
                   L::kIdescDw, ks > 0 ? 1u : 0u);
        }
        tc_commit(bar);
        if (!mbar_wait_bounded(bar, 0)) {
            *abort_flag = 1;
            atomicOr(status, kStatusTimeout);
        }
    }
    __syncthreads();
    tc_fence_after();
    if (!*abort_flag) {
        // this thread's TMEM lane: output i = t of gW, sample t of dZprev
        const uint32_t lane_base = tmem + ((uint32_t)(warp * 32) << 16);
        float* pw = part_w + ((size_t)blockIdx.x * kHid + t) * K;
#pragma unroll 1
        for (int cb = 0; cb < K; cb += 32) {
            float v[32];
            tc_ld32(lane_base + 128u + (uint32_t)cb, v);
#pragma unroll
            for (int q = 0; q < 32; q += 4)
                *reinterpret_cast<float4*>(pw + cb + q) = make_float4(v[q], v[q + 1], v[q + 2], v[q + 3]);
        }
        // bias gradient: the samples of row t of dZ^T, in sample order
        float sbias = 0.f;
        for (int c = 0; c < 16; ++c) {
            const uint4 v = *reinterpret_cast<const uint4*>(sm + L::kADw + sw_off(t, c >> 3, c & 7, kBkBlock));
            const __nv_bfloat162* e = reinterpret_cast<const __nv_bfloat162*>(&v);
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const float2 f = __bfloat1622float2(e[q]);
                sbias += f.x;
                sbias += f.y;
            }
        }
        part_b[(size_t)blockIdx.x * kHid + t] = sbias;
        if (want_dx) {
            const size_t o = (size_t)(base + t) * kHid;
#pragma unroll 1
            for (int cb = 0; cb < 128; cb += 32) {
                float v[32];
                tc_ld32(lane_base + (uint32_t)cb, v);   // every lane of the warp takes part
                if (t < rows) {
#pragma unroll
                    for (int q = 0; q < 32; q += 8) {
                        const uint4 zv = *reinterpret_cast<const uint4*>(zprev + o + cb + q);
                        const __nv_bfloat162* ze = reinterpret_cast<const __nv_bfloat162*>(&zv);
                        uint32_t u[4];
#pragma unroll
                        for (int k = 0; k < 4; ++k) {
                            const float2 zf = __bfloat1622float2(ze[k]);
                            u[k] = bf16_pair(v[q + 2 * k] * gelu_grad(zf.x),
                                             v[q + 2 * k + 1] * gelu_grad(zf.y));
                        }
                        *reinterpret_cast<uint4*>(dzprev + o + cb + q) = make_uint4(u[0], u[1], u[2], u[3]);
                    }
                }
            }
        }
    }
    // the MMAs of an aborted CTA may still write TMEM: wait once more (bounded)
    tc_fence_before();
    __syncthreads();
    if (t == 0 && *abort_flag) mbar_wait_bounded(bar, 0);
    __syncthreads();
    tc_fence_after();
    if (warp == 0) tc_dealloc(tmem, 256);
}

struct SurrogateRowParams {
    Weights w;
    const Tile* tiles;
    int tile_begin, tile_end;
    const uint16_t* ev_bin;
    const float* ev_e;
    const int* q_pix;
    const float* g8;       // [A][nq][8]
    float* rows;
    int64_t row_base;
    int row_stride;
    const float* lam;      // may be null
    int lam_stride;
    const uint16_t* ev_real;   // realisation of each sorted event, or null (tile's own)
    float* ypart;
    int64_t ypart_stride;
    int* status;
    int n, A, B, W, nq, nqt;
    float h, bin_w;
    float mu_line[LMMEW_MAX_LINES];
    float e_line[LMMEW_MAX_LINES];
    // recorded energies that single scatter of line w can reach: between its
    // backscatter energy and E_w, widened by 8 energy-resolution sigmas
    float reach_lo[LMMEW_MAX_LINES], reach_hi[LMMEW_MAX_LINES];
    const float* rho;
    // coarse-grid form: the columns are network nodes (node_q: their voxels)
    // and the outputs go to nodebuf [event][n_cols] instead of the rows
    const int* node_q;     // null: the columns are the support voxels
    int n_cols, n_col_tiles;
    float* nodebuf;
    int64_t nodebuf_stride;
};

// The surrogate inside the row pipeline: after k_row wrote the unscattered
// part of every row of a (tile of up to 128 events, 32-voxel tile) unit,
// this kernel adds sum_w max(exp(net(x_w)) - eps, 0) to every (event, voxel)
// and writes the unit's partial forward sums.  Line w's term is evaluated
// only for events whose recorded energy its single scatter can reach (the
// backscatter energy to E_w, widened by kSurrogateReachSigmas energy-
// resolution sigmas); elsewhere it is 0.  Each thread group takes every
// fourth unit; passes of 128 samples: 4 reachable events x 32 voxels, one
// line; the thread that owns a sample adds its part to the row in global
// memory.
__global__ void __launch_bounds__(kTcThreads, 1) k_surrogate_rows(const SurrogateRowParams P) {
    extern __shared__ unsigned char smem_raw[];
    const TcShared S = tc_shared(smem_raw);
    const uint32_t tmem_base = tc_setup(S, P.w);
    const TcGroup G = tc_group(S, tmem_base);
    const float b4 = P.w.p[kOffB4];
    float* Vxy = G.f;                     // [32] voxel centre (x, y), cm
    float* Vg8 = Vxy + 32 * 2;            // [32][8] rho line integrals
    float* Eeu = Vg8 + 32 * 8;            // [128] (recorded energy, bin centre)
    int* Cnt = reinterpret_cast<int*>(G.f + kGrpUnitFloats);   // [W] events per line list
    int* Wcnt = Cnt + LMMEW_MAX_LINES;                          // [W][4] per-warp counts
    uint8_t* Act = reinterpret_cast<uint8_t*>(Wcnt + 4 * LMMEW_MAX_LINES);   // [W][128]
    const int gt = G.gt;
    uint32_t phase = 0;
    const int n_tiles = P.tile_end - P.tile_begin;
    const int n_units = n_tiles * P.n_col_tiles;
    const float half_det = 0.5f * P.B * P.bin_w;
    bool ok = true;
    for (int unit = blockIdx.x * kTcGroups + G.g; unit < n_units && ok;
         unit += gridDim.x * kTcGroups) {
        const Tile T = P.tiles[P.tile_begin + unit / P.n_col_tiles];
        const int qt = unit % P.n_col_tiles;   // column tile: 32 voxels or 32 nodes
        const int nq_here = min(32, P.n_cols - qt * 32);
        group_sync(G.g);   // the group's previous unit is done with the unit data
        if (gt < 32 && gt < nq_here) {
            const int pix = P.q_pix[P.node_q ? P.node_q[qt * 32 + gt] : qt * 32 + gt];
            Vxy[2 * gt] = ((pix % P.n) + 0.5f - 0.5f * P.n) * P.h;
            Vxy[2 * gt + 1] = ((pix / P.n) + 0.5f - 0.5f * P.n) * P.h;
        }
        for (int i = gt; i < 32 * 8; i += kGrpThreads)
            if ((i >> 3) < nq_here) {
                const int col = qt * 32 + (i >> 3);
                const int q = P.node_q ? P.node_q[col] : col;
                Vg8[i] = P.g8[((size_t)T.a * P.nq + q) * 8 + (i & 7)];
            }
        if (gt < T.count) {
            Eeu[2 * gt] = P.ev_e[T.begin + gt];
            Eeu[2 * gt + 1] = -half_det + (P.ev_bin[T.begin + gt] + 0.5f) * P.bin_w;
        }
        // per line, the unit's events whose recorded energy its single
        // scatter can reach, as a compact list (warp ballots + prefix)
        {
            const int lane = gt & 31, wq = gt >> 5;
            const float eh = gt < T.count ? P.ev_e[T.begin + gt] : 0.f;
            for (int wl = 0; wl < P.W; ++wl) {
                const bool f = gt < T.count && eh >= P.reach_lo[wl] && eh <= P.reach_hi[wl];
                const unsigned m = __ballot_sync(0xffffffffu, f);
                if (lane == 0) Wcnt[wl * 4 + wq] = __popc(m);
            }
            group_sync(G.g);
            for (int wl = 0; wl < P.W; ++wl) {
                const bool f = gt < T.count && eh >= P.reach_lo[wl] && eh <= P.reach_hi[wl];
                const unsigned m = __ballot_sync(0xffffffffu, f);
                int off = 0;
                for (int i = 0; i < wq; ++i) off += Wcnt[wl * 4 + i];
                if (f) Act[wl * 128 + off + __popc(m & ((1u << lane) - 1u))] = (uint8_t)gt;
                if (gt == 0)
                    Cnt[wl] = Wcnt[wl * 4] + Wcnt[wl * 4 + 1] + Wcnt[wl * 4 + 2] + Wcnt[wl * 4 + 3];
            }
        }
        group_sync(G.g);
        const float th = 6.283185307179586f * T.a / P.A;
        float ca, sa;
        sincosf(th, &sa, &ca);
        // passes of 4 listed events x 32 voxels, one line at a time; the
        // thread that owns a sample adds its scatter part to the row (passes
        // are ordered by the group barriers inside each network evaluation)
        for (int wl = 0; wl < P.W && ok; ++wl) {
            const int n_act = Cnt[wl];
            const uint8_t* act = Act + wl * 128;
            for (int c = 0; c < (n_act + 3) / 4 && ok; ++c) {
                // the 32 inputs of the thread's own sample gt (listed event
                // 4c + gt / 32, voxel gt mod 32) into row gt of X, built in one
                // piece so the geometry shared by the last 16 is formed once
                {
                    const int slot = c * 4 + (gt >> 5), ql = gt & 31;
                    float f[32];
                    if (slot < n_act && ql < nq_here) {
                        const int e = act[slot];
                        surrogate_features(Vxy[2 * ql], Vxy[2 * ql + 1], ca, sa, Eeu[2 * e + 1],
                                           Eeu[2 * e], wl, P.e_line[wl], P.mu_line[wl],
                                           Vg8 + ql * 8, P.rho, P.n, P.h, f);
                    } else {
#pragma unroll
                        for (int i = 0; i < 32; ++i) f[i] = 0.f;
                    }
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        uint32_t u[4];
#pragma unroll
                        for (int i = 0; i < 4; ++i) {
                            const __nv_bfloat162 t =
                                __floats2bfloat162_rn(f[8 * j + 2 * i], f[8 * j + 2 * i + 1]);
                            u[i] = *reinterpret_cast<const uint32_t*>(&t);
                        }
                        *reinterpret_cast<uint4*>(S.base + G.h + sw_chunk(gt, 0, j)) =
                            make_uint4(u[0], u[1], u[2], u[3]);
                    }
                }
                tc_input_constants(S, G);
                fence_async_smem();
                group_sync(G.g);
                float o = 0.f;
                ok = tc_network<false>(S, G, phase, b4, &o, P.status);
                const int slot = c * 4 + (gt >> 5), ql = gt & 31;
                if (ok && slot < n_act && ql < nq_here) {
                    const float v = __expf(o) - kSurrogateEps;
                    if (v > 0.f) {
                        const size_t e = (size_t)(T.begin + act[slot] - P.row_base);
                        if (P.node_q)
                            P.nodebuf[e * P.nodebuf_stride + qt * 32 + ql] += v;
                        else
                            P.rows[e * P.row_stride + qt * 32 + ql] += v;
                    }
                }
            }
        }
        if (!ok) break;
        group_sync(G.g);   // the group's row updates are visible to the whole group
        if (P.lam && !P.node_q && gt < T.count) {
            const int rr = P.ev_real ? (int)P.ev_real[T.begin + gt] : T.r;
            const float* lam = P.lam + (size_t)rr * P.lam_stride;
            const float* row = P.rows + (size_t)(T.begin + gt - P.row_base) * P.row_stride + qt * 32;
            float s = 0.f;
            for (int ql = 0; ql < nq_here; ++ql) s = fmaf(lam[qt * 32 + ql], row[ql], s);
            P.ypart[(size_t)qt * P.ypart_stride + (T.begin + gt - P.row_base)] = s;
        }
    }
    tc_teardown(S, G, tmem_base, phase);
}

// Coarse-grid surrogate: each voxel's scatter part is the weighted sum of
// its nodes' network outputs (weights summing to 1); it is added to the
// voxel's row, then the forward partial sum of every 32-voxel tile is
// formed in a fixed order.  One warp per event, a lane per voxel of the tile.
__global__ void __launch_bounds__(256) k_interp_rows(const int4* inode, const float4* iw,
                                                     const float* nodebuf, int64_t nb_stride,
                                                     float* rows, int row_stride, int64_t count,
                                                     int nq, const float* lam, int lam_stride,
                                                     const uint16_t* ev_real, int64_t row_base,
                                                     float* ypart, int64_t ypart_stride) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t e = (int64_t)blockIdx.x * 8 + warp;
    const int qt = blockIdx.y;
    const int q = qt * 32 + lane;
    if (e >= count) return;   // the whole warp leaves together
    float v = 0.f;
    if (q < nq) {
        const int4 id = inode[q];
        const float4 w = iw[q];
        const float* nb = nodebuf + e * nb_stride;
        float sct = w.x * nb[id.x];
        if (id.y >= 0) sct = fmaf(w.y, nb[id.y], sct);
        if (id.z >= 0) sct = fmaf(w.z, nb[id.z], sct);
        if (id.w >= 0) sct = fmaf(w.w, nb[id.w], sct);
        float* r = rows + e * row_stride + q;
        v = *r + sct;
        *r = v;
    }
    if (lam) {
        const float* lm = lam + (ev_real ? (size_t)ev_real[row_base + e] * lam_stride : 0);
        float p = q < nq ? lm[q] * v : 0.f;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) p += __shfl_xor_sync(0xffffffffu, p, o);
        if (lane == 0) ypart[(size_t)qt * ypart_stride + e] = p;
    }
}

}  // namespace mlp
}  // namespace lmmew

// ---------------------------------------------------------------------------
// Host side: the surrogate object and its C ABI.
using lmmew::mlp::bf16;
namespace M = lmmew::mlp;

struct lm_surrogate {
    float* p = nullptr;      // FP32 master parameters [kParams]
    float* m1 = nullptr;     // Adam moments
    float* m2 = nullptr;
    float* grad = nullptr;
    bf16* W1 = nullptr;      // BF16 copies used by the tensor-core kernels
    bf16* W2 = nullptr;
    bf16* W3 = nullptr;
    int64_t step = 0;
    void* scratch = nullptr;
    size_t scratch_bytes = 0;
    int* status = nullptr;   // device status word of the tensor-core forward
};

namespace lmmew {

const void* surrogate_weights(const lm_surrogate* s, void* out_weights) {
    mlp::Weights* w = reinterpret_cast<mlp::Weights*>(out_weights);
    w->W1 = s->W1;
    w->W2 = s->W2;
    w->W3 = s->W3;
    w->p = s->p;
    return out_weights;
}

// Shared-memory opt-in of the surrogate kernels.  The attribute belongs to the
// current device, so it is set once per device the library runs on.
int surrogate_kernel_attrs() {
    static std::atomic<unsigned long long> done{0};
    int dev = 0;
    LMMEW_CUDA(cudaGetDevice(&dev));
    const unsigned long long bit = 1ull << (dev & 63);
    if (done.load() & bit) return LMMEW_OK;
    LMMEW_CUDA(cudaFuncSetAttribute(mlp::k_tc_forward<false>,
                                    cudaFuncAttributeMaxDynamicSharedMemorySize, (int)mlp::kTcSmem));
    LMMEW_CUDA(cudaFuncSetAttribute(mlp::k_tc_forward<true>,
                                    cudaFuncAttributeMaxDynamicSharedMemorySize, (int)mlp::kTcSmem));
    LMMEW_CUDA(cudaFuncSetAttribute(mlp::k_surrogate_rows,
                                    cudaFuncAttributeMaxDynamicSharedMemorySize, (int)mlp::kTcSmem));
    LMMEW_CUDA(cudaFuncSetAttribute(mlp::k_tc_back_layer<mlp::kHid>,
                                    cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)mlp::BackTc<mlp::kHid>::kSmem));
    LMMEW_CUDA(cudaFuncSetAttribute(mlp::k_tc_back_layer<mlp::kIn>,
                                    cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)mlp::BackTc<mlp::kIn>::kSmem));
    done.fetch_or(bit);
    return LMMEW_OK;
}

// Nodes of the coarse-grid surrogate: the support voxels at even pixel
// coordinates that some voxel interpolates from, and the support voxels
// without any such neighbour (their own node).  Voxel (ix, iy) takes the
// bilinear weights of the even-coordinate corners around it, (ix & ~1,
// iy & ~1) to (+2, +2), keeps the corners in the support and renormalises
// the weights to sum 1.  Built on the host once per handle.
int build_coarse_nodes(lm_handle* h) {
    if (h->d_node_q) return LMMEW_OK;
    const int n = h->mc.n, nq = h->mc.nq;
    std::vector<int> q_pix(nq);
    LMMEW_CUDA(cudaMemcpy(q_pix.data(), h->d_q_pix, sizeof(int) * nq, cudaMemcpyDeviceToHost));
    std::vector<int> q_of_pix((size_t)n * n, -1);
    for (int q = 0; q < nq; ++q) q_of_pix[q_pix[q]] = q;
    std::vector<int> node_of_q(nq, -1), node_q;
    auto node_for = [&](int q) {
        if (node_of_q[q] < 0) {
            node_of_q[q] = (int)node_q.size();
            node_q.push_back(q);
        }
        return node_of_q[q];
    };
    std::vector<int4> idx(nq);
    std::vector<float4> wt(nq);
    for (int q = 0; q < nq; ++q) {
        const int ix = q_pix[q] % n, iy = q_pix[q] / n;
        const int st = h->coarse_stride;
        const int x0 = ix - ix % st, y0 = iy - iy % st;
        const double tx = (double)(ix - x0) / st, ty = (double)(iy - y0) / st;
        const int cx[4] = {x0, x0 + st, x0, x0 + st}, cy[4] = {y0, y0, y0 + st, y0 + st};
        const double w0[4] = {(1 - tx) * (1 - ty), tx * (1 - ty), (1 - tx) * ty, tx * ty};
        int cq[4];
        double sum = 0.0;
        for (int k = 0; k < 4; ++k) {
            cq[k] = (w0[k] > 0.0 && cx[k] < n && cy[k] < n) ? q_of_pix[(size_t)cy[k] * n + cx[k]] : -1;
            if (cq[k] >= 0) sum += w0[k];
        }
        int ni[4] = {-1, -1, -1, -1};
        float nw[4] = {0.f, 0.f, 0.f, 0.f};
        if (sum <= 0.0) {
            ni[0] = node_for(q);
            nw[0] = 1.f;
        } else {
            int j = 0;
            for (int k = 0; k < 4; ++k)
                if (cq[k] >= 0) {
                    ni[j] = node_for(cq[k]);
                    nw[j] = (float)(w0[k] / sum);
                    ++j;
                }
        }
        idx[q] = make_int4(ni[0], ni[1], ni[2], ni[3]);
        wt[q] = make_float4(nw[0], nw[1], nw[2], nw[3]);
    }
    const int nn = (int)node_q.size();
    if (cudaMalloc(&h->d_node_q, sizeof(int) * nn) != cudaSuccess ||
        cudaMalloc(&h->d_interp_node, sizeof(int4) * nq) != cudaSuccess ||
        cudaMalloc(&h->d_interp_w, sizeof(float4) * nq) != cudaSuccess) {
        cudaGetLastError();
        cudaFree(h->d_node_q);
        cudaFree(h->d_interp_node);
        cudaFree(h->d_interp_w);
        h->d_node_q = nullptr;
        h->d_interp_node = nullptr;
        h->d_interp_w = nullptr;
        return set_error(LMMEW_ERR_OOM, "cannot allocate the coarse-grid surrogate tables");
    }
    LMMEW_CUDA(cudaMemcpy(h->d_node_q, node_q.data(), sizeof(int) * nn, cudaMemcpyHostToDevice));
    LMMEW_CUDA(cudaMemcpy(h->d_interp_node, idx.data(), sizeof(int4) * nq, cudaMemcpyHostToDevice));
    LMMEW_CUDA(cudaMemcpy(h->d_interp_w, wt.data(), sizeof(float4) * nq, cudaMemcpyHostToDevice));
    h->n_nodes = nn;
    return LMMEW_OK;
}

int surrogate_prepare(lm_handle* h, int64_t max_events, cudaStream_t st) {
    if (h->scatter_model != LMMEW_SCATTER_SURROGATE_COARSE) return LMMEW_OK;
    const size_t need = sizeof(float) * (size_t)std::max<int64_t>(max_events, 1) * h->n_nodes;
    if (h->scratch_nodes.bytes >= need) return LMMEW_OK;
    if (h->scratch_nodes.ptr) {
        LMMEW_CUDA(cudaStreamSynchronize(st));
        cudaFree(h->scratch_nodes.ptr);
        h->scratch_nodes.ptr = nullptr;
        h->scratch_nodes.bytes = 0;
    }
    if (cudaMalloc(&h->scratch_nodes.ptr, need) != cudaSuccess) {
        cudaGetLastError();
        return set_error(LMMEW_ERR_OOM, "cannot allocate the coarse-grid surrogate outputs");
    }
    h->scratch_nodes.bytes = need;
    return LMMEW_OK;
}

int launch_surrogate_rows(lm_handle* h, const RowLaunch& L, cudaStream_t st) {
    const bool coarse = h->scatter_model == LMMEW_SCATTER_SURROGATE_COARSE;
    const int n_cols = coarse ? h->n_nodes : h->mc.nq;
    const int n_col_tiles = (n_cols + 31) / 32;
    const int n_units = (L.tile_end - L.tile_begin) * n_col_tiles;
    if (n_units <= 0) return LMMEW_OK;
    int rc = surrogate_kernel_attrs();
    if (rc != LMMEW_OK) return rc;
    const int64_t count = L.n_events;   // events of the row block
    const size_t node_bytes = sizeof(float) * (size_t)std::max<int64_t>(count, 0) * h->n_nodes;
    if (coarse && h->scratch_nodes.bytes < node_bytes)
        return set_error(LMMEW_ERR_INVALID_ARG,
                         "coarse-grid surrogate outputs not prepared for this row block");
    mlp::SurrogateRowParams P;
    surrogate_weights(h->surrogate, &P.w);
    P.tiles = L.tiles;
    P.tile_begin = L.tile_begin;
    P.tile_end = L.tile_end;
    P.ev_bin = L.ev_bin;
    P.ev_e = L.ev_e;
    P.q_pix = h->d_q_pix;
    P.g8 = h->d_g8;
    P.status = h->d_status;
    P.rows = L.rows;
    P.row_base = L.row_base;
    P.row_stride = L.row_stride;
    P.lam = L.lam_v;
    P.lam_stride = L.lam_stride;
    P.ev_real = L.ev_real;
    P.ypart = L.ypart;
    P.ypart_stride = L.ypart_stride;
    P.n = h->mc.n;
    P.A = h->mc.A;
    P.B = h->mc.B;
    P.W = h->mc.W;
    P.nq = h->mc.nq;
    P.nqt = h->mc.nqt;
    P.h = (float)h->mc.h;
    P.bin_w = (float)h->mc.bin_w;
    const ModelConst& m = h->mc;
    const double fwhm_to_sigma = 1.0 / (2.0 * std::sqrt(2.0 * std::log(2.0)));
    auto sigma_e = [&](double e) {
        return m.fwhm_frac * e * std::pow(e / m.e_ref, m.expo) * fwhm_to_sigma;
    };
    for (int w = 0; w < LMMEW_MAX_LINES; ++w) {
        P.mu_line[w] = (float)h->mu_line[w];
        P.e_line[w] = (float)m.line_e[w];
        const double ew = m.line_e[w] > 0.0 ? m.line_e[w] : 1.0;
        const double e_back = ew / (1.0 + 2.0 * ew / kElectronRestKeV);   // Compton, 180 degrees
        P.reach_lo[w] = (float)(e_back - kSurrogateReachSigmas * sigma_e(e_back));
        P.reach_hi[w] = (float)(ew + kSurrogateReachSigmas * sigma_e(ew));
    }
    P.rho = h->d_rho;
    P.node_q = coarse ? h->d_node_q : nullptr;
    P.n_cols = n_cols;
    P.n_col_tiles = n_col_tiles;
    P.nodebuf = coarse ? (float*)h->scratch_nodes.ptr : nullptr;
    P.nodebuf_stride = h->n_nodes;
    if (coarse) LMMEW_CUDA(cudaMemsetAsync(P.nodebuf, 0, node_bytes, st));
    const int grid = std::min((n_units + mlp::kTcGroups - 1) / mlp::kTcGroups, h->sm_count);
    mlp::k_surrogate_rows<<<grid, mlp::kTcThreads, mlp::kTcSmem, st>>>(P);
    ++h->launches;
    LMMEW_CUDA(cudaGetLastError());
    if (coarse && count > 0) {
        dim3 g((unsigned)((count + 7) / 8), (unsigned)h->mc.nqt);
        mlp::k_interp_rows<<<g, 256, 0, st>>>(h->d_interp_node, h->d_interp_w, P.nodebuf, h->n_nodes,
                                              L.rows, L.row_stride, count, h->mc.nq, L.lam_v,
                                              L.lam_stride, L.ev_real, L.row_base, L.ypart,
                                              L.ypart_stride);
        ++h->launches;
        LMMEW_CUDA(cudaGetLastError());
    }
    return LMMEW_OK;
}

namespace {

int ensure_scratch(lm_surrogate* s, size_t bytes) {
    if (s->scratch_bytes >= bytes) return LMMEW_OK;
    LMMEW_CUDA(cudaDeviceSynchronize());
    cudaFree(s->scratch);
    s->scratch = nullptr;
    s->scratch_bytes = 0;
    if (cudaMalloc(&s->scratch, bytes) != cudaSuccess) {
        cudaGetLastError();
        return set_error(LMMEW_ERR_OOM, "cannot allocate surrogate scratch");
    }
    s->scratch_bytes = bytes;
    return LMMEW_OK;
}

int refresh_bf16(lm_surrogate* s, cudaStream_t st) {
    M::k_to_bf16<<<(M::kHid * M::kIn + 255) / 256, 256, 0, st>>>(s->p + M::kOffW1, M::kHid * M::kIn, s->W1);
    M::k_to_bf16<<<(M::kHid * M::kHid + 255) / 256, 256, 0, st>>>(s->p + M::kOffW2, M::kHid * M::kHid, s->W2);
    M::k_to_bf16<<<(M::kHid * M::kHid + 255) / 256, 256, 0, st>>>(s->p + M::kOffW3, M::kHid * M::kHid, s->W3);
    LMMEW_CUDA(cudaGetLastError());
    return LMMEW_OK;
}

int set_attrs() { return surrogate_kernel_attrs(); }

int sm_count() {
    int dev = 0, count = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&count, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return 1;
    return count > 0 ? count : 1;
}

// Full-batch gradient of mean squared error over n samples of BF16 inputs
// xb; grad (device) receives dL/dp.  Optionally the loss (host).
int gradient(lm_surrogate* s, const bf16* xb, const float* t, const float* v, int64_t n,
             double* loss, cudaStream_t st) {
    const int64_t n_cta = (n + M::kTile - 1) / M::kTile;
    const int64_t npad = n_cta * M::kTile;
    size_t off = 0;
    auto take = [&](size_t bytes) { size_t o = off; off += (bytes + 255) / 256 * 256; return o; };
    const size_t o_out = take(sizeof(float) * npad);
    const size_t o_z = take(sizeof(bf16) * 3 * npad * M::kHid);
    const size_t o_d3 = take(sizeof(bf16) * npad * M::kHid);
    const size_t o_d2 = take(sizeof(bf16) * npad * M::kHid);
    const size_t o_d1 = take(sizeof(bf16) * npad * M::kHid);
    const size_t o_pw1 = take(sizeof(float) * n_cta * M::kHid * M::kIn);
    const size_t o_pb1 = take(sizeof(float) * n_cta * M::kHid);
    const size_t o_pw2 = take(sizeof(float) * n_cta * M::kHid * M::kHid);
    const size_t o_pb2 = take(sizeof(float) * n_cta * M::kHid);
    const size_t o_pw3 = take(sizeof(float) * n_cta * M::kHid * M::kHid);
    const size_t o_pb3 = take(sizeof(float) * n_cta * M::kHid);
    const size_t o_po = take(sizeof(float) * n_cta * (M::kHid + 1));
    const size_t o_mse = take(sizeof(double) * 256);
    int rc = ensure_scratch(s, off);
    if (rc != LMMEW_OK) return rc;
    rc = set_attrs();
    if (rc != LMMEW_OK) return rc;
    char* base = (char*)s->scratch;
    float* out = (float*)(base + o_out);
    bf16* z = (bf16*)(base + o_z);
    bf16* d3 = (bf16*)(base + o_d3);
    bf16* d2 = (bf16*)(base + o_d2);
    bf16* d1 = (bf16*)(base + o_d1);
    M::Weights w{s->W1, s->W2, s->W3, s->p};
    // forward on the tensor cores, keeping the hidden pre-activations
    // one 128-sample tile per group; as many CTAs as SMs allow
    const int fwd_grid = (int)std::min<int64_t>(n_cta, sm_count());
    M::k_tc_forward<true><<<fwd_grid, M::kTcThreads, M::kTcSmem, st>>>(w, xb, n, out, s->status, z);
    M::k_back_out<<<(unsigned)n_cta, M::kThreads, 0, st>>>(s->p, out, t, v, z + 2 * n * M::kHid, n,
                                                          1.f / (float)n, d3, (float*)(base + o_po));
    // hidden layers 3, 2, 1 on the tensor cores
    M::k_tc_back_layer<M::kHid><<<(unsigned)n_cta, 128, M::BackTc<M::kHid>::kSmem, st>>>(
        d3, z + n * M::kHid, nullptr, s->W3, n, (float*)(base + o_pw3), (float*)(base + o_pb3), d2,
        s->status);
    M::k_tc_back_layer<M::kHid><<<(unsigned)n_cta, 128, M::BackTc<M::kHid>::kSmem, st>>>(
        d2, z, nullptr, s->W2, n, (float*)(base + o_pw2), (float*)(base + o_pb2), d1, s->status);
    M::k_tc_back_layer<M::kIn><<<(unsigned)n_cta, 128, M::BackTc<M::kIn>::kSmem, st>>>(
        d1, nullptr, xb, s->W1, n, (float*)(base + o_pw1), (float*)(base + o_pb1), nullptr,
        s->status);
    M::k_reduce_grad<<<(M::kParams + 255) / 256, 256, 0, st>>>(
        (float*)(base + o_pw1), (float*)(base + o_pb1), (float*)(base + o_pw2), (float*)(base + o_pb2),
        (float*)(base + o_pw3), (float*)(base + o_pb3), (float*)(base + o_po), (int)n_cta, s->grad);
    LMMEW_CUDA(cudaGetLastError());
    if (loss) {
        double* mse = (double*)(base + o_mse);
        M::k_mse<<<64, 256, 0, st>>>(out, t, v, n, mse);
        double host[64];
        LMMEW_CUDA(cudaMemcpyAsync(host, mse, sizeof(host), cudaMemcpyDeviceToHost, st));
        LMMEW_CUDA(cudaStreamSynchronize(st));
        double sum = 0.0;
        for (int i = 0; i < 64; ++i) sum += host[i];
        *loss = sum / (double)n;
    }
    return LMMEW_OK;
}

int to_bf16_inputs(lm_surrogate* s, const float* x, int64_t n, bf16** xb, size_t extra_off,
                   cudaStream_t st) {
    (void)s;
    M::k_to_bf16<<<(unsigned)((n * M::kIn + 255) / 256), 256, 0, st>>>(x, n * M::kIn, *xb);
    LMMEW_CUDA(cudaGetLastError());
    (void)extra_off;
    return LMMEW_OK;
}

uint64_t splitmix_host(uint64_t& state) {
    uint64_t z = (state += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

}  // namespace
}  // namespace lmmew

using namespace lmmew;

extern "C" {

int lm_surrogate_param_count(void) { return M::kParams; }

int lm_surrogate_create(uint64_t seed, lm_surrogate** out) {
    if (!out) return set_error(LMMEW_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    lm_surrogate* s = new lm_surrogate();
    const size_t pb = sizeof(float) * M::kParams;
    if (cudaMalloc(&s->p, pb) != cudaSuccess || cudaMalloc(&s->m1, pb) != cudaSuccess ||
        cudaMalloc(&s->m2, pb) != cudaSuccess || cudaMalloc(&s->grad, pb) != cudaSuccess ||
        cudaMalloc(&s->W1, sizeof(bf16) * M::kHid * M::kIn) != cudaSuccess ||
        cudaMalloc(&s->W2, sizeof(bf16) * M::kHid * M::kHid) != cudaSuccess ||
        cudaMalloc(&s->W3, sizeof(bf16) * M::kHid * M::kHid) != cudaSuccess ||
        cudaMalloc(&s->status, sizeof(int)) != cudaSuccess) {
        cudaGetLastError();
        lm_surrogate_destroy(s);
        return set_error(LMMEW_ERR_OOM, "cannot allocate the surrogate");
    }
    // Xavier-uniform weights, zero biases, output bias at a typical log value
    std::vector<float> p(M::kParams, 0.f);
    uint64_t st = seed;
    auto uni = [&](float lim) {
        const double u = (double)(splitmix_host(st) >> 11) * (1.0 / 9007199254740992.0);
        return (float)((2.0 * u - 1.0) * lim);
    };
    const float l1 = std::sqrt(6.f / (M::kIn + M::kHid)), l2 = std::sqrt(6.f / (2 * M::kHid)),
                l4 = std::sqrt(6.f / (M::kHid + 1));
    for (int i = 0; i < M::kHid * M::kIn; ++i) p[M::kOffW1 + i] = uni(l1);
    for (int i = 0; i < M::kHid * M::kHid; ++i) p[M::kOffW2 + i] = uni(l2);
    for (int i = 0; i < M::kHid * M::kHid; ++i) p[M::kOffW3 + i] = uni(l2);
    for (int i = 0; i < M::kHid; ++i) p[M::kOffW4 + i] = uni(l4);
    p[M::kOffB4] = -10.f;
    int rc = LMMEW_OK;
    if (cudaMemcpy(s->p, p.data(), pb, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemset(s->m1, 0, pb) != cudaSuccess || cudaMemset(s->m2, 0, pb) != cudaSuccess ||
        cudaMemset(s->status, 0, sizeof(int)) != cudaSuccess)
        rc = set_error(LMMEW_ERR_CUDA, "surrogate initialisation");
    if (rc == LMMEW_OK) rc = refresh_bf16(s, 0);
    if (rc == LMMEW_OK && cudaDeviceSynchronize() != cudaSuccess)
        rc = set_error(LMMEW_ERR_CUDA, "surrogate initialisation");
    if (rc != LMMEW_OK) {
        lm_surrogate_destroy(s);
        return rc;
    }
    *out = s;
    return LMMEW_OK;
}

int lm_surrogate_destroy(lm_surrogate* s) {
    if (!s) return LMMEW_OK;
    cudaFree(s->p);
    cudaFree(s->m1);
    cudaFree(s->m2);
    cudaFree(s->grad);
    cudaFree(s->W1);
    cudaFree(s->W2);
    cudaFree(s->W3);
    cudaFree(s->scratch);
    cudaFree(s->status);
    delete s;
    return LMMEW_OK;
}

int lm_surrogate_get_params(const lm_surrogate* s, float* host_out) {
    if (!s || !host_out) return set_error(LMMEW_ERR_INVALID_ARG, "NULL argument");
    LMMEW_CUDA(cudaMemcpy(host_out, s->p, sizeof(float) * M::kParams, cudaMemcpyDeviceToHost));
    int status = 0;
    LMMEW_CUDA(cudaMemcpy(&status, s->status, sizeof(int), cudaMemcpyDeviceToHost));
    if (status & kStatusTimeout) {
        LMMEW_CUDA(cudaMemset(s->status, 0, sizeof(int)));
        return set_error(LMMEW_ERR_TIMEOUT, "a tensor-core wait of an earlier forward pass ran out");
    }
    return LMMEW_OK;
}

int lm_surrogate_set_params(lm_surrogate* s, const float* host_in) {
    if (!s || !host_in) return set_error(LMMEW_ERR_INVALID_ARG, "NULL argument");
    LMMEW_CUDA(cudaMemcpy(s->p, host_in, sizeof(float) * M::kParams, cudaMemcpyHostToDevice));
    int rc = refresh_bf16(s, 0);
    if (rc != LMMEW_OK) return rc;
    LMMEW_CUDA(cudaDeviceSynchronize());
    return LMMEW_OK;
}

int lm_surrogate_forward(lm_surrogate* s, const float* x, int64_t n, float* out, lm_stream stream) {
    if (!s || (n > 0 && (!x || !out))) return set_error(LMMEW_ERR_INVALID_ARG, "NULL argument");
    if (n <= 0) return LMMEW_OK;
    cudaStream_t st = (cudaStream_t)stream;
    int rc = ensure_scratch(s, sizeof(bf16) * (size_t)n * M::kIn + 256);
    if (rc != LMMEW_OK) return rc;
    rc = set_attrs();
    if (rc != LMMEW_OK) return rc;
    bf16* xb = (bf16*)s->scratch;
    rc = to_bf16_inputs(s, x, n, &xb, 0, st);
    if (rc != LMMEW_OK) return rc;
    M::Weights w{s->W1, s->W2, s->W3, s->p};
    const int64_t tiles = (n + 127) / 128;
    const unsigned grid = (unsigned)std::min<int64_t>((tiles + M::kTcGroups - 1) / M::kTcGroups, sm_count());
    M::k_tc_forward<false><<<grid, M::kTcThreads, M::kTcSmem, st>>>(w, xb, n, out, s->status);
    LMMEW_CUDA(cudaGetLastError());
    return LMMEW_OK;
}

int lm_surrogate_gradient(lm_surrogate* s, const float* x, const float* target,
                          const float* weight, int64_t n, float* grad_out, double* loss_out,
                          lm_stream stream) {
    if (!s || !x || !target || !grad_out || n <= 0)
        return set_error(LMMEW_ERR_INVALID_ARG, "bad argument");
    cudaStream_t st = (cudaStream_t)stream;
    bf16* xb = nullptr;
    if (cudaMalloc(&xb, sizeof(bf16) * (size_t)n * M::kIn) != cudaSuccess) {
        cudaGetLastError();
        return set_error(LMMEW_ERR_OOM, "cannot allocate the BF16 inputs");
    }
    int rc = to_bf16_inputs(s, x, n, &xb, 0, st);
    if (rc == LMMEW_OK) rc = gradient(s, xb, target, weight, n, loss_out, st);
    if (rc == LMMEW_OK &&
        cudaMemcpyAsync(grad_out, s->grad, sizeof(float) * M::kParams, cudaMemcpyDeviceToDevice,
                        st) != cudaSuccess)
        rc = set_error(LMMEW_ERR_CUDA, "gradient copy");
    cudaStreamSynchronize(st);
    cudaFree(xb);
    return rc;
}

int lm_surrogate_train(lm_surrogate* s, const float* x, const float* target, int64_t n, int steps,
                       int batch, float lr, float weight_power, uint64_t seed,
                       double* loss_history, lm_stream stream) {
    if (!s || !x || !target || n <= 0 || steps < 0 || batch < 1 || batch > (1 << 20) ||
        !(lr > 0.f) || !(weight_power >= 0.f) || !(weight_power <= 64.f))
        return set_error(LMMEW_ERR_INVALID_ARG, "bad argument");
    if (n >= (int64_t(1) << 32)) return set_error(LMMEW_ERR_INVALID_ARG, "too many samples");
    cudaStream_t st = (cudaStream_t)stream;
    bf16* xall = nullptr;
    bf16* xb = nullptr;
    float* tb = nullptr;
    uint32_t* idx = nullptr;
    float* vall = nullptr;
    float* vb = nullptr;
    const bool weighted = weight_power > 0.f;
    if (cudaMalloc(&xall, sizeof(bf16) * (size_t)n * M::kIn) != cudaSuccess ||
        cudaMalloc(&xb, sizeof(bf16) * (size_t)batch * M::kIn) != cudaSuccess ||
        cudaMalloc(&tb, sizeof(float) * batch) != cudaSuccess ||
        cudaMalloc(&idx, sizeof(uint32_t) * batch) != cudaSuccess ||
        (weighted && (cudaMalloc(&vall, sizeof(float) * (size_t)n) != cudaSuccess ||
                      cudaMalloc(&vb, sizeof(float) * batch) != cudaSuccess))) {
        cudaGetLastError();
        cudaFree(xall); cudaFree(xb); cudaFree(tb); cudaFree(idx); cudaFree(vall); cudaFree(vb);
        return set_error(LMMEW_ERR_OOM, "cannot allocate training buffers");
    }
    int rc = to_bf16_inputs(s, x, n, &xall, 0, st);
    if (weighted) M::k_train_weights<<<1, 1024, 0, st>>>(target, n, weight_power, vall);
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    for (int k = 0; k < steps && rc == LMMEW_OK; ++k) {
        M::k_batch_indices<<<(batch + 255) / 256, 256, 0, st>>>(seed, (uint64_t)s->step, batch,
                                                                (uint64_t)n, idx);
        M::k_gather_batch_rows<<<(batch * (M::kIn / 8) + 255) / 256, 256, 0, st>>>(
            xall, target, vall, idx, batch, xb, tb, vb);
        double loss = 0.0;
        rc = gradient(s, xb, tb, vb, batch, loss_history ? &loss : nullptr, st);
        if (rc != LMMEW_OK) break;
        if (loss_history) loss_history[k] = loss;
        s->step += 1;
        const float c1 = 1.f - std::pow(b1, (float)s->step), c2 = 1.f - std::pow(b2, (float)s->step);
        M::k_adam<<<(M::kParams + 255) / 256, 256, 0, st>>>(s->p, s->m1, s->m2, s->grad, lr, b1, b2,
                                                          eps, c1, c2, s->W1, s->W2, s->W3);
        if (cudaGetLastError() != cudaSuccess) rc = set_error(LMMEW_ERR_CUDA, "training step");
    }
    cudaStreamSynchronize(st);
    cudaFree(xall); cudaFree(xb); cudaFree(tb); cudaFree(idx); cudaFree(vall); cudaFree(vb);
    return rc;
}

}  // extern "C"
