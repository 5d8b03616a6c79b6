// The hot kernel: system-matrix rows of the path model computed on the fly
// (paper Eq. Aj_expansion with Eq. s_p for n = 0 and n = 1; Algorithm 1's
// K_SumAjKernel), fused with the per-tile partial forward projection.
//
//   a_j[q] = sum_w alpha_w [ s_prim(a,w,q) C_q(b) g(E_hat; E_w)
//                            + sum_p s(a,w,q,p) C_p(b) g(E_hat; E'(a,w,q,p)) ]
//
// Work unit = (tile of up to 32 EPL events of one angle, tile of 32 voxels),
// EPL = 1, 2 or 4 events per lane (the tile size is autotuned); the
// persistent CTAs take units from a counter as they finish the last one.  The
// CTA streams the angle's scatter-path tables for its 32 voxels and the
// collimator rows of the tile's bins, 32 scatter points per stage (points in
// the angle's ascending detector-coordinate order, only the run of chunks
// whose collimator probability for the tile's bins is non-zero, and in the
// run's first and last chunk only its 4-point groups inside the run), from
// global memory into shared memory with bulk asynchronous copies (TMA engine,
// cp.async.bulk + mbarrier, double buffered).  Each of the 8 warps owns 4
// voxels; each lane owns EPL events, so a table entry read from shared memory
// is a broadcast that feeds EPL events, and the collimator value of an
// (event, point) pair feeds every voxel and line.  Per scatter term, in the
// square-root form of the energy Gaussian:
//   d = sr E_hat + m;  arg = d d + nlh;  term = ex2(-arg)   (FMA, FMA, MUFU)
// with sr = sqrt(log2(e) / 2) / sigma_E(E'), m = -sr E' and
// nlh = -log2(alpha s / (sqrt(2 pi) sigma_E(E'))) precomputed in FP64, so a
// term costs two FMA-pipe operations before its exponential (plus the line
// sum and the collimator product, one more per term amortised) instead of
// three; the FP32 arithmetic runs on packed pairs of scatter points (f32x2),
// one instruction covering two terms.  Sums are hierarchical: per stage,
// per unit, then across warps in a fixed order, so results are
// deterministic.  Every mbarrier wait is bounded in time; a wait that runs
// out sets the status word and the CTA stops cleanly.
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <algorithm>

#include "lmmew_internal.cuh"

namespace lmmew {
namespace {

__device__ __forceinline__ float fast_ex2(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

struct RowParams {
    const float* tab;     // [A][nqt][npc][3][W][kQT][kPC]: nlh, sr, m
    const float* tabh;    // reduced-precision form: [A][nqt][npc]{-E' f32 [W][kQT][kPC],
                          //   (lh - base, nk) halves [W][kQT][kPC/4][8]}
    const float* tscale;  // [A][nqt][npc] 2^base of each block (reduced precision)
    const float* cs;      // [A][npc][B][kCPad]
    const int2* crange;   // [A][B] run of points with non-zero collimator probability
    unsigned long long* term_counter;   // if set: exponentials evaluated for valid (event, voxel)
    int* work;            // units handed out beyond the first gridDim.x (zero at launch)
    const float* cv;      // [A][B][nq]
    const float* prim;    // [A][W][nq]
    const Tile* tiles;
    int tile_begin, tile_end;
    const uint16_t* ev_bin;
    const float* ev_e;
    const float* lam;     // [nq] (per realisation, lam_stride apart) or null
    int lam_stride;
    const uint16_t* ev_real;   // realisation of each sorted event, or null (tile's own)
    int unit_order;       // 0: tile-major, 1: voxel-tile-major work units
    int skip_scatter;     // 1: unscattered terms only
    float* rows;          // or null
    int64_t row_base;
    int row_stride;
    float* ypart;         // [nqt][ypart_stride] or null
    int64_t ypart_stride;
    int* status;
    int W, B, nq, nqt, npc, np;
    uint32_t stage_bytes;   // bytes of one pipeline stage in shared memory
    uint32_t tab_stage_bytes;
    LineConst lc;
};

// 2^-(d^2 + nlh) with d = sr e_hat + m, for one event and two scatter points.
__device__ __forceinline__ f32x2 term2(f32x2 eh2, f32x2 sr, f32x2 m, f32x2 nlh) {
    const f32x2 d = fma2(sr, eh2, m);
    const f32x2 a = fma2(d, d, nlh);
    float a0, a1;
    upk(a, a0, a1);
    return pk(fast_ex2(-a0), fast_ex2(-a1));
}

// Packed half-precision arithmetic for the reduced-precision form: PREC 1 =
// FP16 (f16x2), PREC 2 = BF16 (bf16x2).  Values travel as .b32 pairs.
template <int PREC> struct Half;
template <> struct Half<1> {
    static __device__ __forceinline__ uint32_t cvt(float lo, float hi) {
        uint32_t r;
        asm("cvt.rn.f16x2.f32 %0, %1, %2;" : "=r"(r) : "f"(hi), "f"(lo));
        return r;
    }
    static __device__ __forceinline__ uint32_t mul(uint32_t a, uint32_t b) {
        uint32_t r;
        asm("mul.rn.f16x2 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(b));
        return r;
    }
    static __device__ __forceinline__ uint32_t fma(uint32_t a, uint32_t b, uint32_t c) {
        uint32_t r;
        asm("fma.rn.f16x2 %0, %1, %2, %3;" : "=r"(r) : "r"(a), "r"(b), "r"(c));
        return r;
    }
    static __device__ __forceinline__ uint32_t add(uint32_t a, uint32_t b) {
        uint32_t r;
        asm("add.rn.f16x2 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(b));
        return r;
    }
    static __device__ __forceinline__ uint32_t ex2(uint32_t a) {
        uint32_t r;
        asm("ex2.approx.f16x2 %0, %1;" : "=r"(r) : "r"(a));
        return r;
    }
    static __device__ __forceinline__ f32x2 widen(uint32_t h) {
        float lo, hi;
        asm("{\n .reg .b16 l, h;\n mov.b32 {l, h}, %2;\n cvt.f32.f16 %0, l;\n cvt.f32.f16 %1, h;\n}"
            : "=f"(lo), "=f"(hi) : "r"(h));
        return pk(lo, hi);
    }
};
template <> struct Half<2> {
    static __device__ __forceinline__ uint32_t cvt(float lo, float hi) {
        uint32_t r;
        asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(r) : "f"(hi), "f"(lo));
        return r;
    }
    static __device__ __forceinline__ uint32_t mul(uint32_t a, uint32_t b) {
        uint32_t r;
        asm("mul.rn.bf16x2 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(b));
        return r;
    }
    static __device__ __forceinline__ uint32_t fma(uint32_t a, uint32_t b, uint32_t c) {
        uint32_t r;
        asm("fma.rn.bf16x2 %0, %1, %2, %3;" : "=r"(r) : "r"(a), "r"(b), "r"(c));
        return r;
    }
    static __device__ __forceinline__ uint32_t add(uint32_t a, uint32_t b) {
        uint32_t r;
        asm("add.rn.bf16x2 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(b));
        return r;
    }
    static __device__ __forceinline__ uint32_t ex2(uint32_t a) {
        uint32_t r;
        asm("ex2.approx.ftz.bf16x2 %0, %1;" : "=r"(r) : "r"(a));
        return r;
    }
    static __device__ __forceinline__ f32x2 widen(uint32_t h) {
        // a bf16 is the upper half of the FP32 with the same bits
        return pk(__uint_as_float(h << 16), __uint_as_float(h & 0xffff0000u));
    }
};

// One pipeline stage of the FP32 form: the 4-point groups [pq0, pq1) of the
// stage's 32 scatter points (all of them when kFull) x 4 voxels x 4 events
// per lane, all lines.
template <int W, bool kFull, int EPL>
__device__ __forceinline__ void stage_fp32(const unsigned char* sb, int warp, const int* bo,
                                           const f32x2* eh2, f32x2 (*acc2)[4], int pq0, int pq1) {
    constexpr int kTabBytes = 3 * W * kQT * kPC * 4;
    const float* tb = reinterpret_cast<const float*>(sb) + warp * 4 * kPC;
    const float* cr = reinterpret_cast<const float*>(sb + kTabBytes);
    const int lo = kFull ? 0 : pq0, hi = kFull ? kPC / 4 : pq1;
#pragma unroll 4
    for (int pq = lo; pq < hi; ++pq) {
        f32x2 cA[EPL], cB[EPL];
#pragma unroll
        for (int k = 0; k < EPL; ++k) {
            const float4 c4 = *reinterpret_cast<const float4*>(cr + bo[k] * kCPad + pq * 4);
            cA[k] = pk(c4.x, c4.y);
            cB[k] = pk(c4.z, c4.w);
        }
#pragma unroll
        for (int qi = 0; qi < 4; ++qi) {
            const float* tq = tb + qi * kPC + pq * 4;
            f32x2 inA[EPL], inB[EPL];
#pragma unroll
            for (int w = 0; w < W; ++w) {
                const float4 nl = *reinterpret_cast<const float4*>(tq + (0 * W + w) * kQT * kPC);
                const float4 sr = *reinterpret_cast<const float4*>(tq + (1 * W + w) * kQT * kPC);
                const float4 mm = *reinterpret_cast<const float4*>(tq + (2 * W + w) * kQT * kPC);
                const f32x2 nlA = pk(nl.x, nl.y), nlB = pk(nl.z, nl.w);
                const f32x2 srA = pk(sr.x, sr.y), srB = pk(sr.z, sr.w);
                const f32x2 mA = pk(mm.x, mm.y), mB = pk(mm.z, mm.w);
#pragma unroll
                for (int k = 0; k < EPL; ++k) {
                    const f32x2 tA = term2(eh2[k], srA, mA, nlA);
                    const f32x2 tB = term2(eh2[k], srB, mB, nlB);
                    inA[k] = (w == 0) ? tA : add2(inA[k], tA);
                    inB[k] = (w == 0) ? tB : add2(inB[k], tB);
                }
            }
#pragma unroll
            for (int k = 0; k < EPL; ++k) {
                acc2[k][qi] = fma2(cA[k], inA[k], acc2[k][qi]);
                acc2[k][qi] = fma2(cB[k], inB[k], acc2[k][qi]);
            }
        }
    }
}

// One stage of the reduced-precision form.  The difference d = E_hat - E'
// stays FP32; nk*d, the exponent (lh relative to the stage block's largest
// log2 weight) and ex2 run on packed halves, the per-line sum in halves, the
// accumulation in FP32 with the block's scale 2^base folded into the
// collimator factor.
template <int W, int PREC>
__device__ __forceinline__ void stage_half(const unsigned char* sb, int warp, const int* bo,
                                           const f32x2* eh2, float scale, f32x2 (*acc2)[4],
                                           int pq0, int pq1) {
    typedef Half<PREC> H;
    constexpr int kTabBytes = 2 * W * kQT * kPC * 4;
    const float* ep = reinterpret_cast<const float*>(sb) + warp * 4 * kPC;
    const uint4* ln = reinterpret_cast<const uint4*>(sb + W * kQT * kPC * 4) + warp * 4 * (kPC / 4);
    const float* cr = reinterpret_cast<const float*>(sb + kTabBytes);
    const f32x2 sc2 = pk(scale, scale);
#pragma unroll 1
    for (int pq = pq0; pq < pq1; ++pq) {
        f32x2 cA[kEPL], cB[kEPL];
#pragma unroll
        for (int k = 0; k < kEPL; ++k) {
            const float4 c4 = *reinterpret_cast<const float4*>(cr + bo[k] * kCPad + pq * 4);
            cA[k] = mul2(pk(c4.x, c4.y), sc2);
            cB[k] = mul2(pk(c4.z, c4.w), sc2);
        }
#pragma unroll
        for (int qi = 0; qi < 4; ++qi) {
            uint32_t inA[kEPL], inB[kEPL];
#pragma unroll
            for (int w = 0; w < W; ++w) {
                const float4 ne =
                    *reinterpret_cast<const float4*>(ep + (w * kQT) * kPC + qi * kPC + pq * 4);
                const uint4 hl = ln[(w * kQT) * (kPC / 4) + qi * (kPC / 4) + pq];
                const f32x2 neA = pk(ne.x, ne.y), neB = pk(ne.z, ne.w);
#pragma unroll
                for (int k = 0; k < kEPL; ++k) {
                    float d0, d1;
                    upk(add2(eh2[k], neA), d0, d1);
                    uint32_t dh = H::cvt(d0, d1);
                    const uint32_t eA = H::ex2(H::fma(H::mul(hl.z, dh), dh, hl.x));
                    upk(add2(eh2[k], neB), d0, d1);
                    dh = H::cvt(d0, d1);
                    const uint32_t eB = H::ex2(H::fma(H::mul(hl.w, dh), dh, hl.y));
                    inA[k] = (w == 0) ? eA : H::add(inA[k], eA);
                    inB[k] = (w == 0) ? eB : H::add(inB[k], eB);
                }
            }
#pragma unroll
            for (int k = 0; k < kEPL; ++k) {
                acc2[k][qi] = fma2(cA[k], H::widen(inA[k]), acc2[k][qi]);
                acc2[k][qi] = fma2(cB[k], H::widen(inB[k]), acc2[k][qi]);
            }
        }
    }
}

template <int W, int PREC, int EPL>
__global__ void __launch_bounds__(kRowThreads, 2) k_row(const RowParams P) {
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ __align__(8) uint64_t bars[2];
    __shared__ int s_abort;
    __shared__ int s_unit;

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const uint32_t bar0 = smem_addr(&bars[0]), bar1 = smem_addr(&bars[1]);
    if (tid == 0) {
        mbar_init(bar0, 1);
        mbar_init(bar1, 1);
        mbar_fence_init();
        s_abort = 0;
    }
    __syncthreads();

    const int n_tiles = P.tile_end - P.tile_begin;
    const int n_units = n_tiles * P.nqt;
    constexpr int kTabBlock = (PREC == 0 ? 3 : 2) * W * kQT * kPC;   // 4-byte words per (a, qt, pc)
    constexpr uint32_t kTabBytes = kTabBlock * 4u;
    uint32_t g = 0;                                       // pipeline stages issued so far

    // each CTA starts on unit blockIdx.x and then takes the next unhanded
    // unit from the counter, so CTAs that drew lighter units take more
    for (int unit = blockIdx.x; unit < n_units;) {
        const Tile T = P.tiles[P.tile_begin + (P.unit_order ? unit % n_tiles : unit / P.nqt)];
        const int qt = P.unit_order ? unit / n_tiles : unit % P.nqt;
        const float* lam = P.lam ? P.lam + (size_t)T.r * P.lam_stride : nullptr;
        const int b_lo = T.b_lo_hi >> 16, b_hi = T.b_lo_hi & 0xffff;
        const uint32_t c_bytes = (uint32_t)(b_hi - b_lo + 1) * kCPad * 4u;

        float eh[EPL];
        f32x2 eh2[EPL];
        int bo[EPL];
#pragma unroll
        for (int k = 0; k < EPL; ++k) {
            const int e = k * 32 + lane;
            const bool v = e < T.count;
            eh[k] = v ? P.ev_e[T.begin + e] : 0.f;
            eh2[k] = pk(eh[k], eh[k]);
            bo[k] = v ? (int)P.ev_bin[T.begin + e] - b_lo : 0;
        }
        // two partial sums per (event, voxel): even and odd scatter points
        f32x2 acc2[EPL][4];
#pragma unroll
        for (int k = 0; k < EPL; ++k)
#pragma unroll
            for (int i = 0; i < 4; ++i) acc2[k][i] = 0ull;

        // scatter points whose collimator probability is non-zero for some bin
        // of the tile: a contiguous run [p_lo, p_hi) in this angle's point
        // order, staged as whole chunks and evaluated in groups of 4 points;
        // every other term is an exact zero and is not evaluated
        int p_lo = P.np, p_hi = 0;
        for (int b = b_lo; b <= b_hi && !P.skip_scatter; ++b) {
            const int2 r = P.crange[(size_t)T.a * P.B + b];
            if (r.y > r.x) {
                p_lo = min(p_lo, r.x);
                p_hi = max(p_hi, r.y);
            }
        }
        const int pc_lo = p_lo < p_hi ? p_lo / kPC : 0;
        const int pc_hi = p_lo < p_hi ? (p_hi + kPC - 1) / kPC : 0;
        if (P.term_counter && tid == 0) {
            const int nq_here = min(kQT, P.nq - qt * kQT);
            const int np_here = p_lo < p_hi ? min((p_hi + 3) & ~3, P.np) - (p_lo & ~3) : 0;
            atomicAdd(P.term_counter,
                      (unsigned long long)T.count * nq_here * W * (unsigned long long)(np_here + 1));
        }
        if (pc_lo < pc_hi) {
            const float* tab_u = (PREC == 0 ? P.tab : P.tabh) +
                                 ((size_t)T.a * P.nqt + qt) * P.npc * (size_t)kTabBlock;
            const float* scale_u = P.tscale + ((size_t)T.a * P.nqt + qt) * P.npc;
            const float* cs_u = P.cs + ((size_t)T.a * P.npc * P.B + b_lo) * kCPad;
            auto issue = [&](int pc, uint32_t gs) {
                const int buf = gs & 1;
                const uint32_t bar = buf ? bar1 : bar0;
                const uint32_t dst = smem_addr(smem + buf * P.stage_bytes);
                mbar_expect_tx(bar, kTabBytes + c_bytes);
                bulk_g2s(dst, tab_u + (size_t)pc * kTabBlock, kTabBytes, bar);
                bulk_g2s(dst + kTabBytes, cs_u + (size_t)pc * P.B * kCPad, c_bytes, bar);
            };
            if (tid == 0) issue(pc_lo, g);
            for (int pc = pc_lo; pc < pc_hi; ++pc, ++g) {
                if (tid == 0 && pc + 1 < pc_hi) issue(pc + 1, g + 1);
                const int buf = g & 1;
                const bool ok = mbar_wait_bounded(buf ? bar1 : bar0, (g >> 1) & 1);
                if (!ok) s_abort = 1;
                if (ok) {
                    const unsigned char* sb = smem + buf * P.stage_bytes;
                    // 4-point groups of this chunk inside the run
                    const int pq0 = pc == pc_lo ? (p_lo - pc * kPC) >> 2 : 0;
                    const int pq1 = pc == pc_hi - 1 ? (p_hi - pc * kPC + 3) >> 2 : kPC / 4;
                    if constexpr (PREC == 0) {
                        if (pq0 == 0 && pq1 == kPC / 4)
                            stage_fp32<W, true, EPL>(sb, warp, bo, eh2, acc2, 0, kPC / 4);
                        else
                            stage_fp32<W, false, EPL>(sb, warp, bo, eh2, acc2, pq0, pq1);
                    } else {
                        static_assert(PREC == 0 || EPL == kEPL, "reduced precision uses 128-event tiles");
                        stage_half<W, PREC>(sb, warp, bo, eh2, scale_u[pc], acc2, pq0, pq1);
                    }
                }
                __syncthreads();
                if (s_abort) {
                    if (tid == 0) {
                        atomicOr(P.status, kStatusTimeout);
                        // let the copies still in flight land before the CTA exits
                        mbar_wait_bounded((g & 1) ? bar1 : bar0, (g >> 1) & 1);
                        if (pc + 1 < pc_hi)
                            mbar_wait_bounded(((g + 1) & 1) ? bar1 : bar0, ((g + 1) >> 1) & 1);
                    }
                    return;
                }
            }
        }

        float acc[EPL][4];
#pragma unroll
        for (int k = 0; k < EPL; ++k)
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                float lo, hi;
                upk(acc2[k][i], lo, hi);
                acc[k][i] = lo + hi;
            }

        // unscattered paths
        {
            const int b_base = T.a * P.B + b_lo;
#pragma unroll
            for (int qi = 0; qi < 4; ++qi) {
                const int q = qt * kQT + warp * 4 + qi;
                if (q < P.nq) {
#pragma unroll
                    for (int k = 0; k < EPL; ++k) {
                        if (k * 32 + lane < T.count) {
                            float s = 0.f;
#pragma unroll
                            for (int w = 0; w < W; ++w) {
                                const float d = eh[k] - P.lc.e[w];
                                const float gw = P.lc.norm[w] * fast_ex2(P.lc.nk[w] * d * d);
                                s = fmaf(P.prim[((size_t)T.a * W + w) * P.nq + q], gw, s);
                            }
                            acc[k][qi] = fmaf(P.cv[((size_t)(b_base + bo[k])) * P.nq + q], s, acc[k][qi]);
                        }
                    }
                }
            }
        }

        // transpose through shared memory: tile [32 EPL events][32 voxels]
        float* tt = reinterpret_cast<float*>(smem);
#pragma unroll
        for (int k = 0; k < EPL; ++k)
#pragma unroll
            for (int qi = 0; qi < 4; ++qi) tt[(k * 32 + lane) * 33 + warp * 4 + qi] = acc[k][qi];
        __syncthreads();
        if (P.rows) {
            for (int i = tid; i < 32 * EPL * kQT; i += kRowThreads) {
                const int e = i >> 5, ql = i & 31;
                const int q = qt * kQT + ql;
                if (e < T.count && q < P.nq)
                    P.rows[(size_t)(T.begin + e - P.row_base) * P.row_stride + q] = tt[e * 33 + ql];
            }
        }
        if (lam && tid < T.count) {
            const int e = tid;
            const float* le =
                P.ev_real ? P.lam + (size_t)P.ev_real[T.begin + e] * P.lam_stride : lam;
            float s = 0.f;
            const int qmax = min(kQT, P.nq - qt * kQT);
            for (int ql = 0; ql < qmax; ++ql) s = fmaf(le[qt * kQT + ql], tt[e * 33 + ql], s);
            P.ypart[(size_t)qt * P.ypart_stride + (T.begin + e - P.row_base)] = s;
        }
        if (tid == 0) s_unit = (int)gridDim.x + atomicAdd(P.work, 1);
        __syncthreads();
        unit = s_unit;
    }
}

typedef void (*RowKernel)(const RowParams);
// Kernel for W lines, scatter precision prec and epl events per lane (tiles
// of 32 epl events).  Tiles of 32 and 64 events exist for the FP32 form with
// up to 4 lines; everything else runs 128-event tiles.
RowKernel row_kernel_for(int W, int prec, int epl = kEPL) {
    if (prec == 0 && W <= 4 && epl == 1) {
        switch (W) {
            case 1: return k_row<1, 0, 1>;
            case 2: return k_row<2, 0, 1>;
            case 3: return k_row<3, 0, 1>;
            default: return k_row<4, 0, 1>;
        }
    }
    if (prec == 0 && W <= 4 && epl == 2) {
        switch (W) {
            case 1: return k_row<1, 0, 2>;
            case 2: return k_row<2, 0, 2>;
            case 3: return k_row<3, 0, 2>;
            default: return k_row<4, 0, 2>;
        }
    }
    if (prec == 1) {
        switch (W) {
            case 1: return k_row<1, 1, kEPL>;
            case 2: return k_row<2, 1, kEPL>;
            case 3: return k_row<3, 1, kEPL>;
            case 4: return k_row<4, 1, kEPL>;
            default: return nullptr;
        }
    }
    if (prec == 2) {
        switch (W) {
            case 1: return k_row<1, 2, kEPL>;
            case 2: return k_row<2, 2, kEPL>;
            case 3: return k_row<3, 2, kEPL>;
            case 4: return k_row<4, 2, kEPL>;
            default: return nullptr;
        }
    }
    switch (W) {
        case 1: return k_row<1, 0, kEPL>;
        case 2: return k_row<2, 0, kEPL>;
        case 3: return k_row<3, 0, kEPL>;
        case 4: return k_row<4, 0, kEPL>;
        case 5: return k_row<5, 0, kEPL>;
        case 6: return k_row<6, 0, kEPL>;
        case 7: return k_row<7, 0, kEPL>;
        default: return k_row<8, 0, kEPL>;
    }
}

}  // namespace

static RowParams make_params(lm_handle* h, const RowLaunch& L, int prec) {
    const ModelConst& m = h->mc;
    RowParams P;
    P.tab = h->d_tab;
    P.tabh = h->d_tabh;
    P.tscale = h->d_tscale;
    P.cs = h->d_cs;
    P.crange = h->d_crange;
    P.cv = h->d_cv;
    P.prim = h->d_prim;
    P.tiles = L.tiles;
    P.tile_begin = L.tile_begin;
    P.tile_end = L.tile_end;
    P.ev_bin = L.ev_bin;
    P.ev_e = L.ev_e;
    P.lam = L.lam_v;
    P.lam_stride = L.lam_stride;
    P.ev_real = L.ev_real;
    P.skip_scatter = L.skip_scatter;
    P.unit_order = h->unit_order;
    P.rows = L.rows;
    P.row_base = L.row_base;
    P.row_stride = L.row_stride;
    P.ypart = L.ypart;
    P.ypart_stride = L.ypart_stride;
    P.status = h->d_status;
    P.W = m.W;
    P.B = m.B;
    P.nq = m.nq;
    P.nqt = m.nqt;
    P.npc = m.npc;
    P.np = m.np;
    P.term_counter = h->prof_on ? h->d_term_counter : nullptr;
    P.work = h->d_work;
    P.tab_stage_bytes = (uint32_t)((prec == 0 ? 3 : 2) * m.W * kQT * kPC * 4);
    uint32_t stage = P.tab_stage_bytes + (uint32_t)(m.B * kCPad * 4);
    const uint32_t tr = kET * 33 * 4;   // epilogue transpose tile
    if (stage < tr) stage = tr;
    P.stage_bytes = (stage + 127u) & ~127u;
    P.lc = h->lc;
    return P;
}

size_t row_smem_bytes(const lm_handle* h) {
    RowParams P = make_params(const_cast<lm_handle*>(h), RowLaunch{}, 0);
    return 2 * (size_t)P.stage_bytes;
}

// Shared-memory cap and occupancy of every precision variant for this model.
int row_kernel_occupancy(lm_handle* h) {
    int dev = 0;
    LMMEW_CUDA(cudaGetDevice(&dev));
    int max_optin = 0;
    LMMEW_CUDA(cudaDeviceGetAttribute(&max_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    LMMEW_CUDA(cudaDeviceGetAttribute(&h->sm_count, cudaDevAttrMultiProcessorCount, dev));
    for (int prec = 0; prec < 3; ++prec) {
        RowKernel kern = row_kernel_for(h->mc.W, prec);
        h->row_blocks[prec] = 0;
        if (!kern) continue;
        const size_t smem = 2 * (size_t)make_params(h, RowLaunch{}, prec).stage_bytes;
        // the cap is per kernel, shared by every handle: allow the device maximum
        cudaFuncAttributes fa;
        LMMEW_CUDA(cudaFuncGetAttributes(&fa, kern));
        const int cap = max_optin - (int)fa.sharedSizeBytes;
        if ((int)smem > cap) {
            if (prec == 0)
                return set_error(LMMEW_ERR_INVALID_ARG,
                                 "lines x bins too large for the row kernel's shared-memory stages");
            continue;
        }
        LMMEW_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, cap));
        // the 32- and 64-event tile kernels of the FP32 form (same stages)
        for (int epl = 1; prec == 0 && epl < kEPL; epl *= 2) {
            RowKernel small = row_kernel_for(h->mc.W, 0, epl);
            if (small == kern) continue;
            cudaFuncAttributes fs;
            LMMEW_CUDA(cudaFuncGetAttributes(&fs, small));
            LMMEW_CUDA(cudaFuncSetAttribute(small, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                            max_optin - (int)fs.sharedSizeBytes));
        }
        int blocks = 0;
        LMMEW_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, kern, kRowThreads, smem));
        h->row_blocks[prec] = blocks > 0 ? blocks : 1;
    }
    h->row_blocks_per_sm = h->row_blocks[0];
    return LMMEW_OK;
}

namespace {

int launch_row_kernel(lm_handle* h, const RowLaunch& L, cudaStream_t st) {
    const int n_units = (L.tile_end - L.tile_begin) * h->mc.nqt;
    if (n_units <= 0) return LMMEW_OK;
    const int prec = h->prec;
    RowParams P = make_params(h, L, prec);
    const int per_sm = h->grid_per_sm > 0 ? std::min(h->grid_per_sm, h->row_blocks[prec])
                                          : h->row_blocks[prec];
    const int grid = std::min(n_units, h->sm_count * per_sm);
    // events per lane: the tiles were cut with L.tile_ev events; the
    // 128-event kernel serves any tile (and every form without small tiles)
    const int epl = L.tile_ev == 32 ? 1 : (L.tile_ev == 64 ? 2 : kEPL);
    LMMEW_CUDA(cudaMemsetAsync(h->d_work, 0, sizeof(int), st));
    row_kernel_for(h->mc.W, prec, epl)<<<grid, kRowThreads, 2 * P.stage_bytes, st>>>(P);
    ++h->launches;
    LMMEW_CUDA(cudaGetLastError());
    return LMMEW_OK;
}

}  // namespace

// Rows of the scatter model in use: exact (both terms in k_row), none
// (unscattered term only) or the learned surrogate (k_row writes the
// unscattered rows, the network adds the scatter part and the forward sums).
int launch_row(lm_handle* h, const RowLaunch& L, cudaStream_t st) {
    if (h->scatter_model == LMMEW_SCATTER_EXACT) return launch_row_kernel(h, L, st);
    RowLaunch U = L;
    U.skip_scatter = 1;
    if (h->scatter_model == LMMEW_SCATTER_NONE) return launch_row_kernel(h, U, st);
    if (!L.rows)
        return set_error(LMMEW_ERR_NOT_IMPLEMENTED, "the surrogate scatter model needs stored rows");
    U.lam_v = nullptr;
    const int rc = launch_row_kernel(h, U, st);
    if (rc != LMMEW_OK) return rc;
    return launch_surrogate_rows(h, L, st);
}

// Reduced-precision tables from the FP32 ones: per (angle, voxel tile, point
// chunk) block, base = largest log2 weight; the block keeps -E' in FP32 and
// (lh - base, nk) as packed halves.
template <int PREC>
__global__ void __launch_bounds__(256) k_half_tables(const float* tab, int W, float* tabh,
                                                     float* tscale) {
    const size_t blk = blockIdx.x;
    const int n = W * kQT * kPC;
    // the FP32 tables hold (nlh, sr, m): lh = -nlh, nk = -sr^2, -E' = m / sr
    const float* src = tab + blk * (size_t)(3 * n);
    float* dst = tabh + blk * (size_t)(2 * n);
    __shared__ float red[256];
    float mx = -3.0e38f;
    for (int i = threadIdx.x; i < n; i += 256) {
        const float v = -src[i];
        if (v > -1.0e29f) mx = fmaxf(mx, v);
    }
    red[threadIdx.x] = mx;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (threadIdx.x < o) red[threadIdx.x] = fmaxf(red[threadIdx.x], red[threadIdx.x + o]);
        __syncthreads();
    }
    const float base = red[0] > -1.0e29f ? red[0] : 0.f;
    if (threadIdx.x == 0) tscale[blk] = red[0] > -1.0e29f ? exp2f(base) : 0.f;
    for (int i = threadIdx.x; i < n; i += 256) {   // -E'
        const float sr = src[n + i];
        dst[i] = sr > 0.f ? src[2 * n + i] / sr : 0.f;
    }
    uint16_t* hl = reinterpret_cast<uint16_t*>(dst + n);
    // layout [W][kQT][kPC/4][8]: lh of 4 points, then nk of the same 4 points
    for (int i = threadIdx.x; i < n; i += 256) {
        const int wq = i / kPC, p = i % kPC, pq = p / 4, pl = p % 4;
        const float lh = -src[i], nk = -src[n + i] * src[n + i];
        const float rel = lh > -1.0e29f ? lh - base : -1.0e30f;
        uint16_t a, b;
        if (PREC == 1) {
            const __half ha = __float2half_rn(rel), hb = __float2half_rn(nk);
            a = *reinterpret_cast<const uint16_t*>(&ha);
            b = *reinterpret_cast<const uint16_t*>(&hb);
        } else {
            const __nv_bfloat16 ha = __float2bfloat16_rn(rel), hb = __float2bfloat16_rn(nk);
            a = *reinterpret_cast<const uint16_t*>(&ha);
            b = *reinterpret_cast<const uint16_t*>(&hb);
        }
        hl[((size_t)wq * (kPC / 4) + pq) * 8 + pl] = a;
        hl[((size_t)wq * (kPC / 4) + pq) * 8 + 4 + pl] = b;
    }
}

int set_precision(lm_handle* h, int prec) {
    if (prec < 0 || prec > 2) return set_error(LMMEW_ERR_INVALID_ARG, "unknown precision");
    if (prec == 0 || h->mc.np == 0) {
        h->prec = 0;
        return LMMEW_OK;
    }
    if (!row_kernel_for(h->mc.W, prec) || h->row_blocks[prec] == 0)
        return set_error(LMMEW_ERR_NOT_IMPLEMENTED,
                         "the reduced-precision form supports up to 4 lines");
    if (h->tabh_prec != prec) {
        const ModelConst& m = h->mc;
        const size_t blocks = (size_t)m.A * m.nqt * m.npc;
        if (!h->d_tabh) {
            if (cudaMalloc(&h->d_tabh, blocks * 2 * m.W * kQT * kPC * 4) != cudaSuccess ||
                cudaMalloc(&h->d_tscale, blocks * sizeof(float)) != cudaSuccess) {
                cudaGetLastError();
                return set_error(LMMEW_ERR_OOM, "cannot allocate reduced-precision tables");
            }
        }
        if (prec == 1)
            k_half_tables<1><<<(unsigned)blocks, 256>>>(h->d_tab, m.W, h->d_tabh, h->d_tscale);
        else
            k_half_tables<2><<<(unsigned)blocks, 256>>>(h->d_tab, m.W, h->d_tabh, h->d_tscale);
        LMMEW_CUDA(cudaGetLastError());
        LMMEW_CUDA(cudaDeviceSynchronize());
        h->tabh_prec = prec;
    }
    h->prec = prec;
    return LMMEW_OK;
}

}  // namespace lmmew
