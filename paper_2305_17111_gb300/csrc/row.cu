// Host side of the row kernel (row_kernel.cuh): launch parameters, the
// shared-memory cap and occupancy of every instantiation, the launch itself,
// the scatter-model dispatch and the reduced-precision tables.
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <algorithm>

#include "row_kernel.cuh"

namespace lmmew {
namespace {

// Kernel for W lines, scatter precision prec and tiles of tile_ev events.
// The FP32 form with up to 4 lines has tiles of 32 and 64 events in the
// VPL = 2 layout (2 and 4 events per lane); everything else runs 128-event
// tiles in the VPL = 4 layout.  With streamed tables (FP32 only) the
// 64-event kernel also serves 32-event tiles.
RowKernel row_kernel_for(int W, int prec, int tile_ev = kET, bool streamed = false) {
    if (prec != 0) return row_kernel_half(W, prec);
    if (streamed)
        return W <= 4 && tile_ev <= 64 ? row_kernel_f32_t64(W, true) : row_kernel_f32_t128(W, true);
    if (W <= 4 && tile_ev == 32) return row_kernel_f32_t32(W);
    if (W <= 4 && tile_ev == 64) return row_kernel_f32_t64(W);
    return row_kernel_f32_t128(W);
}

}  // namespace

static RowParams make_params(lm_handle* h, const RowLaunch& L, int prec) {
    const ModelConst& m = h->mc;
    RowParams P;
    P.tab = h->d_tab;
    P.tab_a0 = h->tab_slots ? h->tab_a0 : 0;
    P.tab_astep = h->tab_slots ? h->tab_astep : 1;
    P.tab_nslots = h->tab_slots ? h->tab_count : h->mc.A;
    P.tabh = h->d_tabh;
    P.tscale = h->d_tscale;
    P.cs = h->d_cs;
    P.crange = h->d_crange;
    P.cv = h->d_cv;
    P.prim = h->d_prim;
    P.tiles = L.tiles;
    P.tile_begin = L.tile_begin;
    P.tile_end = L.tile_end;
    P.range = L.range;
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
        // the 32- and 64-event tile kernels of the FP32 form and the
        // streamed-table kernels (same stages)
        for (int te = 32; prec == 0 && te <= kET; te *= 2) {
            for (int streamed = 0; streamed < 2; ++streamed) {
                RowKernel other = row_kernel_for(h->mc.W, 0, te, streamed != 0);
                if (other == kern) continue;
                cudaFuncAttributes fs;
                LMMEW_CUDA(cudaFuncGetAttributes(&fs, other));
                LMMEW_CUDA(cudaFuncSetAttribute(other, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                max_optin - (int)fs.sharedSizeBytes));
            }
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
    // the tiles were cut with L.tile_ev events; the 128-event kernel serves
    // any tile (and every form without small tiles)
    LMMEW_CUDA(cudaMemsetAsync(h->d_work, 0, sizeof(int), st));
    const bool streamed = h->tab_slots != 0 && prec == 0;
    row_kernel_for(h->mc.W, prec, L.tile_ev, streamed)<<<grid, kRowThreads, 2 * P.stage_bytes, st>>>(P);
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
    if (h->tab_slots)
        return set_error(LMMEW_ERR_NOT_IMPLEMENTED,
                         "the reduced-precision form needs every angle's path tables resident "
                         "(lm_set_table_streaming(h, 0))");
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
