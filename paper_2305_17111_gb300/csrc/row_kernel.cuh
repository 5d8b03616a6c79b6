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
// one instruction covering two terms.  Each tile holds events of one energy
// class, which fixes the lines whose single scatter can reach its recorded
// energies (Tile::lines); only those lines' tables are staged and evaluated,
// the others' terms being below exp(-32) of their own path's peak.  Sums
// are hierarchical: per stage,
// per unit, then across warps in a fixed order, so results are
// deterministic.  Every mbarrier wait is bounded in time; a wait that runs
// out sets the status word and the CTA stops cleanly.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include "lmmew_internal.cuh"

namespace lmmew {

struct RowParams {
    const float* tab;     // [slots][nqt][npc][3][W][kQT][kPC]: nlh, sr, m
    int tab_a0, tab_astep;   // angle a's tables in slot (a - tab_a0) / tab_astep
    int tab_nslots;          // slots holding tables (a unit outside them is skipped and flagged)
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
    const ChunkRange* range;   // if set: tiles [x, y) and row_base z read from the device
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

typedef void (*RowKernel)(const RowParams);

// The row kernel's instantiations, one translation unit each (compiled in
// parallel): FP32 tiles of 32 and 64 events (up to 4 lines), FP32 tiles of
// 128 events (any line count) and the reduced-precision forms (128-event
// tiles, up to 4 lines).  nullptr where a combination does not exist.
// With streamed path tables (`streamed`), the forms that read them index a
// block of angles (RowParams::tab_a0, tab_astep) and check that every tile's
// angle is in it: separate instantiations of the 64- and 128-event kernels,
// so that the resident form's code is left as it is.
RowKernel row_kernel_f32_t32(int W);
RowKernel row_kernel_f32_t64(int W, bool streamed = false);
RowKernel row_kernel_f32_t128(int W, bool streamed = false);
RowKernel row_kernel_half(int W, int prec);

#ifdef LMMEW_ROW_KERNEL_BODY
namespace rowk {


__device__ __forceinline__ float fast_ex2(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}


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
// stage's 32 scatter points (all of them when kFull) x VPL voxels (from the
// stage's local voxel v0) x EPL events per lane, for the W lines staged (the
// tile's reachable lines, in order).
template <int W, bool kFull, int EPL, int VPL>
__device__ __forceinline__ void stage_fp32(const unsigned char* sb, const float* cr, int v0,
                                           const int* bo, const f32x2* eh2, f32x2 (*acc2)[VPL],
                                           int pq0, int pq1) {
    const float* tb = reinterpret_cast<const float*>(sb) + v0 * kPC;
    const int lo = kFull ? 0 : pq0, hi = kFull ? kPC / 4 : pq1;
#pragma unroll 2
    for (int pq = lo; pq < hi; ++pq) {
        f32x2 cA[EPL], cB[EPL];
#pragma unroll
        for (int k = 0; k < EPL; ++k) {
            const float4 c4 = *reinterpret_cast<const float4*>(cr + bo[k] * kCPad + pq * 4);
            cA[k] = pk(c4.x, c4.y);
            cB[k] = pk(c4.z, c4.w);
        }
#pragma unroll
        for (int qi = 0; qi < VPL; ++qi) {
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

// One stage of the reduced-precision form (W = lines staged).  The difference
// d = E_hat - E' stays FP32; nk*d, the exponent (lh relative to the stage
// block's largest log2 weight) and ex2 run on packed halves, the per-line sum
// in halves, the accumulation in FP32 with the block's scale 2^base folded
// into the collimator factor.
template <int W, int PREC>
__device__ __forceinline__ void stage_half(const unsigned char* sb, const float* cr, int warp,
                                           const int* bo, const f32x2* eh2, float scale,
                                           f32x2 (*acc2)[4], int pq0, int pq1) {
    typedef Half<PREC> H;
    const float* ep = reinterpret_cast<const float*>(sb) + warp * 4 * kPC;
    const uint4* ln = reinterpret_cast<const uint4*>(sb + W * kQT * kPC * 4) + warp * 4 * (kPC / 4);
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

// The stage of nw staged lines (1 <= nw <= W): one instantiation per count.
template <int W, int EPL, int VPL>
__device__ __forceinline__ void stage_fp32_n(int nw, bool full, const unsigned char* sb,
                                             const float* cr, int v0, const int* bo,
                                             const f32x2* eh2, f32x2 (*acc2)[VPL], int pq0,
                                             int pq1) {
    if (nw == W) {
        if (full)
            stage_fp32<W, true, EPL, VPL>(sb, cr, v0, bo, eh2, acc2, 0, kPC / 4);
        else
            stage_fp32<W, false, EPL, VPL>(sb, cr, v0, bo, eh2, acc2, pq0, pq1);
        return;
    }
    if constexpr (W > 1)
        stage_fp32_n<W - 1, EPL, VPL>(nw, full, sb, cr, v0, bo, eh2, acc2, pq0, pq1);
}
template <int W, int PREC>
__device__ __forceinline__ void stage_half_n(int nw, const unsigned char* sb, const float* cr,
                                             int warp, const int* bo, const f32x2* eh2,
                                             float scale, f32x2 (*acc2)[4], int pq0, int pq1) {
    if (nw == W) {
        stage_half<W, PREC>(sb, cr, warp, bo, eh2, scale, acc2, pq0, pq1);
        return;
    }
    if constexpr (W > 1)
        stage_half_n<W - 1, PREC>(nw, sb, cr, warp, bo, eh2, scale, acc2, pq0, pq1);
}

// Lane layout: each warp owns 4 voxels of the unit's 32.  VPL = 4: the 32
// lanes take 32 events each and all 4 voxels (EPL events per lane, tiles of
// 32 EPL).  VPL = 2: lanes 0-15 take voxels 0-1 and lanes 16-31 voxels 2-3 of
// the warp, each for 16 events at a time (EPL per lane, tiles of 16 EPL), so
// a table entry read from shared memory (one broadcast per half-warp) feeds
// twice the events of the VPL = 4 layout at the same tile size.
template <int W, int PREC, int EPL, int VPL, bool kStream = false>
__global__ void __launch_bounds__(kRowThreads, 2) k_row(const RowParams P) {
    static_assert(!kStream || PREC == 0, "streamed tables are FP32");
    static_assert(VPL == 4 || VPL == 2, "4 or 2 voxels per lane");
    constexpr int kLanesEv = VPL == 4 ? 32 : 16;     // lanes that share one voxel set
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ __align__(8) uint64_t bars[2];
    __shared__ int s_abort;
    __shared__ int s_unit;

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int ev_lane = lane % kLanesEv;                          // event slot of this lane
    const int v0 = warp * 4 + (VPL == 4 ? 0 : (lane / 16) * 2);   // first voxel of this lane
    const uint32_t bar0 = smem_addr(&bars[0]), bar1 = smem_addr(&bars[1]);
    if (tid == 0) {
        mbar_init(bar0, 1);
        mbar_init(bar1, 1);
        mbar_fence_init();
        s_abort = 0;
    }
    __syncthreads();

    int tile_begin = P.tile_begin, tile_end = P.tile_end;
    int64_t row_base = P.row_base;
    if (P.range) {
        const ChunkRange R = *P.range;
        tile_begin = R.x;
        tile_end = R.y;
        row_base = R.z;
    }
    const int n_tiles = tile_end - tile_begin;
    const int n_units = n_tiles * P.nqt;
    constexpr int kComp = PREC == 0 ? 3 : 2;                         // table components
    constexpr int kTabBlock = kComp * W * kQT * kPC;   // 4-byte words per (a, qt, pc)
    constexpr uint32_t kLineBytes = kQT * kPC * 4u;     // one component of one line
    uint32_t g = 0;                                       // pipeline stages issued so far

    // each CTA starts on unit blockIdx.x and then takes the next unhanded
    // unit from the counter, so CTAs that drew lighter units take more
    for (int unit = blockIdx.x; unit < n_units;) {
        const Tile T = P.tiles[tile_begin + (P.unit_order ? unit % n_tiles : unit / P.nqt)];
        const int qt = P.unit_order ? unit / n_tiles : unit % P.nqt;
        const float* lam = P.lam ? P.lam + (size_t)T.r * P.lam_stride : nullptr;
        const int b_lo = T.b_lo_hi >> 16, b_hi = T.b_lo_hi & 0xffff;
        const uint32_t c_bytes = (uint32_t)(b_hi - b_lo + 1) * kCPad * 4u;
        // lines whose single scatter reaches the tile's energy class, in order
        const int lmask = P.skip_scatter ? 0 : (T.lines & ((1 << W) - 1));
        const int nw = __popc(lmask);
        const uint32_t tab_bytes = (uint32_t)(kComp * nw) * kLineBytes;

        float eh[EPL];
        f32x2 eh2[EPL];
        int bo[EPL];
#pragma unroll
        for (int k = 0; k < EPL; ++k) {
            const int e = k * kLanesEv + ev_lane;
            const bool v = e < T.count;
            eh[k] = v ? P.ev_e[T.begin + e] : 0.f;
            eh2[k] = pk(eh[k], eh[k]);
            bo[k] = v ? (int)P.ev_bin[T.begin + e] - b_lo : 0;
        }
        // two partial sums per (event, voxel): even and odd scatter points
        f32x2 acc2[EPL][VPL];
#pragma unroll
        for (int k = 0; k < EPL; ++k)
#pragma unroll
            for (int i = 0; i < VPL; ++i) acc2[k][i] = 0ull;

        // scatter points whose collimator probability is non-zero for some bin
        // of the tile: a contiguous run [p_lo, p_hi) in this angle's point
        // order (formed with the tiles), staged as whole chunks and evaluated
        // in groups of 4 points; every other term is an exact zero and is not
        // evaluated
        int p_lo = nw > 0 ? T.p_lo : P.np, p_hi = nw > 0 ? T.p_hi : 0;
        // the slot of the angle's tables; with streamed tables a tile whose
        // angle is not in the buffer is a planning error: its scatter terms
        // are not read, and the status word says so
        int slot = T.a;
        if constexpr (kStream) {
            slot = (T.a - P.tab_a0) / P.tab_astep;
            if (nw > 0 && !(slot >= 0 && slot < P.tab_nslots && P.tab_a0 + slot * P.tab_astep == T.a)) {
                if (tid == 0) atomicOr(P.status, kStatusTables);
                p_hi = 0;
                p_lo = P.np;
            }
        }
        const int pc_lo = p_lo < p_hi ? p_lo / kPC : 0;
        const int pc_hi = p_lo < p_hi ? (p_hi + kPC - 1) / kPC : 0;
        if (P.term_counter && tid == 0) {
            const int nq_here = min(kQT, P.nq - qt * kQT);
            const int np_here = p_lo < p_hi ? min((p_hi + 3) & ~3, P.np) - (p_lo & ~3) : 0;
            atomicAdd(P.term_counter, (unsigned long long)T.count * nq_here *
                                          (unsigned long long)(nw * np_here + W));
        }
        if (pc_lo < pc_hi) {
            const float* tab_u = (PREC == 0 ? P.tab : P.tabh) +
                                 ((size_t)slot * P.nqt + qt) * P.npc * (size_t)kTabBlock;
            const float* scale_u = P.tscale + ((size_t)T.a * P.nqt + qt) * P.npc;
            const float* cs_u = P.cs + ((size_t)T.a * P.npc * P.B + b_lo) * kCPad;
            // A stage holds kc point chunks: kc blocks [component][staged
            // line][32 voxels][32 points], then kc blocks of the tile's
            // collimator rows.  With fewer lines staged than the buffer was
            // sized for, more chunks fit (as many as the collimator rows
            // allow), so every stage carries about the same work.
            const int nb = b_hi - b_lo + 1;
            const int kc = max(1, min(W / nw, P.B / nb));
            const int n_chunks = pc_hi - pc_lo;
            const int n_stages = (n_chunks + kc - 1) / kc;
            const uint32_t cr_off = (uint32_t)kc * tab_bytes;
            auto issue = [&](int si, uint32_t gs) {
                const int buf = gs & 1;
                const uint32_t bar = buf ? bar1 : bar0;
                const uint32_t dst = smem_addr(smem + buf * P.stage_bytes);
                const int pc0 = pc_lo + si * kc, cnt = min(kc, pc_hi - pc0);
                mbar_expect_tx(bar, (uint32_t)cnt * (tab_bytes + c_bytes));
                for (int k = 0; k < cnt; ++k) {
                    const float* src = tab_u + (size_t)(pc0 + k) * kTabBlock;
                    const uint32_t dk = dst + (uint32_t)k * tab_bytes;
                    if (nw == W) {
                        bulk_g2s(dk, src, tab_bytes, bar);
                    } else {
                        for (int w = 0, i = 0; w < W; ++w) {
                            if (!((lmask >> w) & 1)) continue;
                            for (int c = 0; c < kComp; ++c)
                                bulk_g2s(dk + (uint32_t)(c * nw + i) * kLineBytes,
                                         src + (size_t)(c * W + w) * (kQT * kPC), kLineBytes, bar);
                            ++i;
                        }
                    }
                    bulk_g2s(dst + cr_off + (uint32_t)k * c_bytes,
                             cs_u + (size_t)(pc0 + k) * P.B * kCPad, c_bytes, bar);
                }
            };
            if (tid == 0) issue(0, g);
            for (int si = 0; si < n_stages; ++si, ++g) {
                if (tid == 0 && si + 1 < n_stages) issue(si + 1, g + 1);
                const int buf = g & 1;
                const bool ok = mbar_wait_bounded(buf ? bar1 : bar0, (g >> 1) & 1);
                if (!ok) s_abort = 1;
                if (ok) {
                    const unsigned char* sb = smem + buf * P.stage_bytes;
                    const int pc0 = pc_lo + si * kc, cnt = min(kc, pc_hi - pc0);
                    for (int k = 0; k < cnt; ++k) {
                        const int pc = pc0 + k;
                        const unsigned char* tk = sb + (uint32_t)k * tab_bytes;
                        const float* ck = reinterpret_cast<const float*>(sb + cr_off + k * c_bytes);
                        // 4-point groups of this chunk inside the run
                        const int pq0 = pc == pc_lo ? (p_lo - pc * kPC) >> 2 : 0;
                        const int pq1 = pc == pc_hi - 1 ? (p_hi - pc * kPC + 3) >> 2 : kPC / 4;
                        if constexpr (PREC == 0 && W > 4) {
                            // more than 4 lines: no energy classes, every line staged
                            if (pq0 == 0 && pq1 == kPC / 4)
                                stage_fp32<W, true, EPL, VPL>(tk, ck, v0, bo, eh2, acc2, 0, kPC / 4);
                            else
                                stage_fp32<W, false, EPL, VPL>(tk, ck, v0, bo, eh2, acc2, pq0, pq1);
                        } else if constexpr (PREC == 0) {
                            stage_fp32_n<W, EPL, VPL>(nw, pq0 == 0 && pq1 == kPC / 4, tk, ck, v0,
                                                      bo, eh2, acc2, pq0, pq1);
                        } else {
                            static_assert(PREC == 0 || (EPL == kEPL && VPL == 4),
                                          "reduced precision uses 128-event tiles");
                            stage_half_n<W, PREC>(nw, tk, ck, warp, bo, eh2, scale_u[pc], acc2, pq0,
                                                  pq1);
                        }
                    }
                }
                __syncthreads();
                if (s_abort) {
                    if (tid == 0) {
                        atomicOr(P.status, kStatusTimeout);
                        // let the copies still in flight land before the CTA exits
                        mbar_wait_bounded((g & 1) ? bar1 : bar0, (g >> 1) & 1);
                        if (si + 1 < n_stages)
                            mbar_wait_bounded(((g + 1) & 1) ? bar1 : bar0, ((g + 1) >> 1) & 1);
                    }
                    return;
                }
            }
        }

        float acc[EPL][VPL];
#pragma unroll
        for (int k = 0; k < EPL; ++k)
#pragma unroll
            for (int i = 0; i < VPL; ++i) {
                float lo, hi;
                upk(acc2[k][i], lo, hi);
                acc[k][i] = lo + hi;
            }

        // unscattered paths
        {
            const int b_base = T.a * P.B + b_lo;
#pragma unroll
            for (int qi = 0; qi < VPL; ++qi) {
                const int q = qt * kQT + v0 + qi;
                if (q < P.nq) {
#pragma unroll
                    for (int k = 0; k < EPL; ++k) {
                        if (k * kLanesEv + ev_lane < T.count) {
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

        // transpose through shared memory: tile [kLanesEv EPL events][32 voxels]
        float* tt = reinterpret_cast<float*>(smem);
#pragma unroll
        for (int k = 0; k < EPL; ++k)
#pragma unroll
            for (int qi = 0; qi < VPL; ++qi) tt[(k * kLanesEv + ev_lane) * 33 + v0 + qi] = acc[k][qi];
        __syncthreads();
        if (P.rows) {
            for (int i = tid; i < kLanesEv * EPL * kQT; i += kRowThreads) {
                const int e = i >> 5, ql = i & 31;
                const int q = qt * kQT + ql;
                if (e < T.count && q < P.nq)
                    P.rows[(size_t)(T.begin + e - row_base) * P.row_stride + q] = tt[e * 33 + ql];
            }
        }
        if (lam && tid < T.count) {
            const int e = tid;
            const float* le =
                P.ev_real ? P.lam + (size_t)P.ev_real[T.begin + e] * P.lam_stride : lam;
            float s = 0.f;
            const int qmax = min(kQT, P.nq - qt * kQT);
            for (int ql = 0; ql < qmax; ++ql) s = fmaf(le[qt * kQT + ql], tt[e * 33 + ql], s);
            P.ypart[(size_t)qt * P.ypart_stride + (T.begin + e - row_base)] = s;
        }
        if (tid == 0) s_unit = (int)gridDim.x + atomicAdd(P.work, 1);
        __syncthreads();
        unit = s_unit;
    }
}

}  // namespace rowk
#endif  // LMMEW_ROW_KERNEL_BODY

}  // namespace lmmew
