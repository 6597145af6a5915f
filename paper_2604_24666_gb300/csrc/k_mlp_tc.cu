// k_mlp_tc.cu -- MLP forward on the 5th-generation tensor cores (tcgen05 +
// TMEM), BF16 or FP16 operands with FP32 accumulation (Sec. 2, Fig. 2d: H
// hidden ReLU layers without bias and a linear output layer).
//
// One persistent CTA per SM walks 128-row tiles of the feature matrix X
// [n x K0]. Warp roles:
//   warp 0     TMA producer: streams X tiles as 128 x 64-element boxes
//              (128-byte swizzle) into a ring of shared-memory stages;
//   warp 1     owns the TMEM accumulator and issues every tcgen05.mma from
//              one thread: layer 0 reads the X stages, layers >= 1 read the
//              activation tile the epilogue wrote back to shared memory;
//   warps 2-5  epilogue: tcgen05.ld of the FP32 accumulator (each warp its
//              32 TMEM lanes = 32 rows), ReLU, conversion to BF16/FP16 and
//              store into the next layer's A operand; the last layer's 16
//              outputs per row go to global memory as FP32.
// All weights stay resident in shared memory for the whole kernel. Operands
// use the canonical K-major layout with 128-byte swizzle: 8-row x 128-byte
// atoms, 16-byte chunk index XOR (row mod 8), atoms 1024 bytes apart.
// Every wait on an mbarrier is bounded in time; on expiry the kernel records
// NIF_ERR_TIMEOUT, drains its own copies and MMAs, frees TMEM and returns.
#include <cuda.h>
#include <cudaTypedefs.h>

#include "nif_internal.cuh"
#include "tc_ptx.cuh"

namespace {

constexpr int kRows = 128;              // MMA M and rows per tile
constexpr int kThreads = 192;           // 6 warps
constexpr uint32_t kStageBytes = kRows * 128;   // one 128 x 64 box of 16-bit elements

struct TcLayout {
    uint32_t x_off, w0_off, wh_off, wo_off, a_off, bar_off, total;
    int stages;   // X ring depth
    int nb0;      // 64-column boxes of X per tile
    int ks0;      // 16-deep k-steps of layer 0
    int nbw;      // 64-column blocks of a W-wide operand
    int ksw;      // k-steps of a W-deep layer
    uint32_t woff[NIF_MAX_LAYERS];   // element offset of each layer in the 16-bit weight copy
};


template <int W>
__global__ void __launch_bounds__(kThreads, 1)
    k_mlp_tc(const __grid_constant__ CUtensorMap xmap, TcLayout lay, const uint16_t* __restrict__ wts,
             int K0, int H, int fmt, int64_t n_max, const uint32_t* __restrict__ n_dev, float* __restrict__ out,
             uint16_t* __restrict__ acts_out, int64_t acts_rows, int acts_ld, int* __restrict__ status) {
    const int64_t n = n_dev ? ((int64_t)*n_dev < n_max ? (int64_t)*n_dev : n_max) : n_max;
    constexpr uint32_t kAccCols = W < 32 ? 32 : W;     // TMEM columns of one accumulator stage
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    const uint64_t wlim = wait_limit(status);   // bound of the work loop's waits
    // 1024-byte alignment of the dynamic buffer (swizzle atoms)
    uint8_t* sm = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int S = lay.stages;
    uint64_t* bars = reinterpret_cast<uint64_t*>(sm + lay.bar_off);
    // bars: [0,S) full, [S,2S) empty, 2S+{0,1} acc_full, 2S+{2,3} act_full, 2S+4 drain
    const int B_ACC = 2 * S, B_ACT = 2 * S + 2, B_DRAIN = 2 * S + 4;
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(sm + lay.bar_off + 8 * (2 * S + 6));
    volatile int* abort_flag = reinterpret_cast<volatile int*>(sm + lay.bar_off + 8 * (2 * S + 6) + 8);
    const int64_t n_tiles = (n + kRows - 1) / kRows;
    const int64_t nt = blockIdx.x < n_tiles ? (n_tiles - blockIdx.x + gridDim.x - 1) / gridDim.x : 0;
    // a CTA without tiles (a chunk whose device count is short or zero) leaves
    // before any barrier, tensor memory or weight load: uniform per CTA
    if (nt == 0) return;

    if (tid == 0) {
        for (int i = 0; i < S; i++) {
            mbar_init(smem_u32(&bars[i]), 1);
            mbar_init(smem_u32(&bars[S + i]), 1);
        }
        mbar_init(smem_u32(&bars[B_ACC]), 1);
        mbar_init(smem_u32(&bars[B_ACC + 1]), 1);
        mbar_init(smem_u32(&bars[B_ACT]), 128);
        mbar_init(smem_u32(&bars[B_ACT + 1]), 128);
        mbar_init(smem_u32(&bars[B_DRAIN]), 1);
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(2 * kAccCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    // resident weights: layer 0 [W x K0], hidden [W x W] x (H-1), output [16 x W]
    load_weight(sm + lay.w0_off, wts + lay.woff[0], W, K0, tid, kThreads);
    for (int l = 1; l < H; l++)
        load_weight(sm + lay.wh_off + (uint32_t)(l - 1) * lay.nbw * W * 128, wts + lay.woff[l], W, W, tid, kThreads);
    load_weight(sm + lay.wo_off, wts + lay.woff[H], 16, W, tid, kThreads);
    fence_async_smem();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;
    const uint32_t a_bytes = (uint32_t)lay.nbw * kRows * 128;   // one activation tile

    if (warp == 0) {
        // ---------------- TMA producer ----------------
        if (lane == 0) {
            asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&xmap)) : "memory");
            int slot = 0;
            uint32_t phase = 0;
            uint32_t issued_parity_mask = 0, issued_mask = 0;
            bool ok = true;
            for (int64_t j = 0; j < nt && ok; j++) {
                int64_t t = blockIdx.x + j * gridDim.x;
                for (int b = 0; b < lay.nb0; b++) {
                    if (!mbar_wait(smem_u32(&bars[S + slot]), phase ^ 1u, abort_flag, status, wlim)) { ok = false; break; }
                    uint32_t fb = smem_u32(&bars[slot]);
                    mbar_expect_tx(fb, kStageBytes);
                    tma_load_2d(smem_u32(sm + lay.x_off + (uint32_t)slot * kStageBytes), &xmap, b * 64,
                                (int)(t * kRows), fb);
                    issued_mask |= 1u << slot;
                    issued_parity_mask = (issued_parity_mask & ~(1u << slot)) | (phase << slot);
                    if (++slot == S) { slot = 0; phase ^= 1u; }
                }
            }
            // drain: every issued copy must have landed before the CTA exits
            for (int i = 0; i < S; i++)
                if (issued_mask >> i & 1u) {
                    volatile int dummy = 0;
                    mbar_wait(smem_u32(&bars[i]), (issued_parity_mask >> i) & 1u, &dummy, status);
                }
        }
    } else if (warp == 1) {
        // ---------------- MMA issuer: tiles in pairs, one TMEM stage each ----------------
        if (lane == 0) {
            const uint32_t id_hid = idesc_f16(fmt, W);
            const uint32_t id_out = idesc_f16(fmt, 16);
            int slot = 0;
            uint32_t phase = 0;
            uint32_t act_par[2] = {0u, 0u};
            bool ok = true;
            for (int64_t j0 = 0; j0 < nt && ok; j0 += 2) {
                const int cnt = nt - j0 < 2 ? (int)(nt - j0) : 2;
                for (int q = 0; q < cnt && ok; q++) {
                    const uint32_t acc = tmem + (uint32_t)q * kAccCols;
                    if (j0 + q >= 2) {      // this stage's accumulator must have been read out
                        if (!mbar_wait(smem_u32(&bars[B_ACT + q]), act_par[q], abort_flag, status, wlim)) { ok = false; break; }
                        act_par[q] ^= 1u;
                        tc_fence_after();
                    }
                    for (int b = 0; b < lay.nb0; b++) {
                        if (!mbar_wait(smem_u32(&bars[slot]), phase, abort_flag, status, wlim)) { ok = false; break; }
                        tc_fence_after();
                        uint32_t base = smem_u32(sm + lay.x_off + (uint32_t)slot * kStageBytes);
                        uint32_t wbase = smem_u32(sm + lay.w0_off + (uint32_t)b * W * 128);
                        for (int jj = 0; jj < 4; jj++) {
                            int ks = b * 4 + jj;
                            if (ks >= lay.ks0) break;
                            mma_f16(acc, sdesc(base + 32 * jj), sdesc(wbase + 32 * jj), id_hid, ks > 0 ? 1u : 0u);
                        }
                        mma_commit(smem_u32(&bars[S + slot]));   // frees the stage when these MMAs finish
                        if (++slot == S) { slot = 0; phase ^= 1u; }
                    }
                    if (!ok) break;
                    mma_commit(smem_u32(&bars[B_ACC + q]));
                }
                // layers 1..H read the activation tile the epilogue wrote for that stage
                for (int l = 1; l <= H && ok; l++) {
                    for (int q = 0; q < cnt && ok; q++) {
                        const uint32_t acc = tmem + (uint32_t)q * kAccCols;
                        if (!mbar_wait(smem_u32(&bars[B_ACT + q]), act_par[q], abort_flag, status, wlim)) { ok = false; break; }
                        act_par[q] ^= 1u;
                        tc_fence_after();
                        const bool last = l == H;
                        uint32_t wb = last ? smem_u32(sm + lay.wo_off)
                                           : smem_u32(sm + lay.wh_off + (uint32_t)(l - 1) * lay.nbw * W * 128);
                        uint32_t ab = smem_u32(sm + lay.a_off + (uint32_t)q * a_bytes);
                        for (int ks = 0; ks < lay.ksw; ks++) {
                            uint32_t blk = (uint32_t)(ks >> 2), jj = (uint32_t)(ks & 3);
                            uint32_t aoff = blk * kRows * 128 + 32 * jj;
                            uint32_t boff = blk * (uint32_t)(last ? 16 : W) * 128 + 32 * jj;
                            mma_f16(acc, sdesc(ab + aoff), sdesc(wb + boff), last ? id_out : id_hid, ks > 0 ? 1u : 0u);
                        }
                        mma_commit(smem_u32(&bars[B_ACC + q]));
                    }
                }
            }
            // all MMAs of this CTA complete before TMEM is released
            mma_commit(smem_u32(&bars[B_DRAIN]));
            volatile int dummy = 0;
            mbar_wait(smem_u32(&bars[B_DRAIN]), 0, &dummy, status);
        }
    } else {
        // ---------------- epilogue (warps 2..5), same pair order ----------------
        const int qw = warp & 3;                  // TMEM lane quarter this warp may access
        const int row = qw * 32 + lane;
        uint32_t acc_par[2] = {0u, 0u};
        bool ok = true;
        for (int64_t j0 = 0; j0 < nt && ok; j0 += 2) {
            const int cnt = nt - j0 < 2 ? (int)(nt - j0) : 2;
            for (int l = 0; l <= H && ok; l++) {
                for (int q = 0; q < cnt; q++) {
                    int got = 0;
                    if (lane == 0) got = mbar_wait(smem_u32(&bars[B_ACC + q]), acc_par[q], abort_flag, status, wlim) ? 1 : 0;
                    got = __shfl_sync(0xffffffffu, got, 0);
                    if (!got) { ok = false; break; }
                    acc_par[q] ^= 1u;
                    tc_fence_after();
                    const uint32_t lane_base = tmem + ((uint32_t)(qw * 32) << 16) + (uint32_t)q * kAccCols;
                    if (l < H) {
                        uint8_t* A = sm + lay.a_off + (uint32_t)q * a_bytes;
                        const int64_t grow = (blockIdx.x + (j0 + q) * gridDim.x) * kRows + row;
                        uint16_t* arow = (acts_out && grow < n) ? acts_out + ((int64_t)l * acts_rows + grow) * acts_ld : nullptr;
                        float v[32];
#pragma unroll
                        for (int c0 = 0; c0 < W; c0 += 32) {
                            tmem_ld32(lane_base + (uint32_t)c0, v);
#pragma unroll
                            for (int c = 0; c < 32; c += 8) {
                                uint4 pk;
                                pk.x = pack2(fmaxf(v[c], 0.f), fmaxf(v[c + 1], 0.f), fmt);
                                pk.y = pack2(fmaxf(v[c + 2], 0.f), fmaxf(v[c + 3], 0.f), fmt);
                                pk.z = pack2(fmaxf(v[c + 4], 0.f), fmaxf(v[c + 5], 0.f), fmt);
                                pk.w = pack2(fmaxf(v[c + 6], 0.f), fmaxf(v[c + 7], 0.f), fmt);
                                *reinterpret_cast<uint4*>(A + swz_off(row, c0 + c, kRows)) = pk;
                                if (arow) *reinterpret_cast<uint4*>(arow + c0 + c) = pk;   // saved for the backward
                            }
                        }
                        fence_async_smem();
                    } else {
                        float v[16];
                        tmem_ld16(lane_base, v);
                        int64_t t = blockIdx.x + (j0 + q) * gridDim.x;
                        int64_t grow = t * kRows + row;
                        if (grow < n) {
                            float4* o = reinterpret_cast<float4*>(out + grow * NIF_OUT);
                            o[0] = make_float4(v[0], v[1], v[2], v[3]);
                            o[1] = make_float4(v[4], v[5], v[6], v[7]);
                            o[2] = make_float4(v[8], v[9], v[10], v[11]);
                            o[3] = make_float4(v[12], v[13], v[14], v[15]);
                        }
                    }
                    tc_fence_before();
                    mbar_arrive(smem_u32(&bars[B_ACT + q]));
                }
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(2 * kAccCols) : "memory");
    }
}

// ---------------------------------------------------------------------------
// Backward of the MLP on tensor cores (the dX chain):
//   dY_H = S * dL/dout,   dY_l = (dY_{l+1} W_{l+1}) * [act_l > 0],   dX_0 = dY_0 W_0,
// with S the loss scale. Every product is D = A B^T with A = dY (K-major, in
// shared memory) and B = W^T, read from a transposed 16-bit copy of the
// weights so that it is K-major too. dX_0 (FP32, in_dim wide) is produced in
// TMEM chunks of at most 256 columns. The 16-bit dY of every layer is written
// out ([H+1][n_pad][ld]) for the weight gradients; activations are read from
// the forward's [H][n_pad][ld] copy.
//
// Hand-off protocol per tile (act_ready counts the 128 epilogue threads):
//   epilogue: write dY_H, arrive | per layer: wait acc, mask, write dY, arrive |
//             per dX_0 chunk: wait acc, store, arrive unless it is the last
//   MMA:      per layer and per chunk: wait act_ready, issue, commit acc_full
// so arrivals and waits alternate strictly on both barriers (the first
// arrival of a tile follows the read of the previous tile's last chunk).
// ---------------------------------------------------------------------------
constexpr int kStg = 36;                 // row stride (floats) of an epilogue warp's 32 x 32 staging tile

struct TcBwdLayout {
    uint32_t wt0_off, wth_off, wto_off, a_off, st_off, bar_off, total;
    int nbw, ksw;
    uint32_t wtoff[NIF_MAX_LAYERS];
};

__device__ __forceinline__ float unpack16(uint16_t v, int fmt) {
    if (fmt == 1) return __bfloat162float(__ushort_as_bfloat16(v));
    return __half2float(__ushort_as_half(v));
}

template <int W>
__global__ void __launch_bounds__(kThreads, 1)
    k_mlp_tc_bwd(TcBwdLayout lay, const uint16_t* __restrict__ wt, int in_dim, int H, int fmt, int64_t n_max,
                 int64_t n_pad, int ld, const uint32_t* __restrict__ n_dev, const float* __restrict__ dout,
                 const uint16_t* __restrict__ acts, const float* __restrict__ scale_dev,
                 uint16_t* __restrict__ dys, float* __restrict__ dx, int* __restrict__ status) {
    constexpr uint32_t kCols = 256;
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    const uint64_t wlim = wait_limit(status);   // bound of the work loop's waits
    uint8_t* sm = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    uint64_t* bars = reinterpret_cast<uint64_t*>(sm + lay.bar_off);   // 0 acc_full, 1 act_ready, 2 drain
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(sm + lay.bar_off + 32);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(sm + lay.bar_off + 40);
    const int64_t n = n_dev ? ((int64_t)*n_dev < n_max ? (int64_t)*n_dev : n_max) : n_max;
    const int64_t n_tiles = (n + kRows - 1) / kRows;
    if ((int64_t)blockIdx.x >= n_tiles) return;   // no tile for this CTA: leave before any setup
    const int n_chunks = (in_dim + (int)kCols - 1) / (int)kCols;
    if (tid == 0) {
        mbar_init(smem_u32(&bars[0]), 1);
        mbar_init(smem_u32(&bars[1]), 128);
        mbar_init(smem_u32(&bars[2]), 1);
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(kCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    // resident transposed weights: W_0^T [in_dim x W], W_l^T [W x W], W_H^T [W x 16]
    load_weight(sm + lay.wt0_off, wt + lay.wtoff[0], in_dim, W, tid, kThreads);
    for (int l = 1; l < H; l++)
        load_weight(sm + lay.wth_off + (uint32_t)(l - 1) * lay.nbw * W * 128, wt + lay.wtoff[l], W, W, tid, kThreads);
    load_weight(sm + lay.wto_off, wt + lay.wtoff[H], W, 16, tid, kThreads);
    fence_async_smem();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;
    const float S = *scale_dev;

    if (warp == 1) {
        if (lane == 0) {
            const uint32_t id_w = idesc_f16(fmt, W);
            uint32_t act_par = 0;
            bool ok = true;
            const uint32_t ab = smem_u32(sm + lay.a_off);
            for (int64_t t = blockIdx.x; t < n_tiles && ok; t += gridDim.x) {
                // layers H .. 1: D = dY_l W_l  (B = W_l^T, K = out_l)
                for (int l = H; l >= 1; l--) {
                    if (!mbar_wait(smem_u32(&bars[1]), act_par, abort_flag, status, wlim)) { ok = false; break; }
                    act_par ^= 1u;
                    tc_fence_after();
                    const int ks_n = l == H ? 1 : lay.ksw;
                    const uint32_t wb = l == H ? smem_u32(sm + lay.wto_off)
                                               : smem_u32(sm + lay.wth_off + (uint32_t)(l - 1) * lay.nbw * W * 128);
                    for (int ks = 0; ks < ks_n; ks++) {
                        uint32_t blk = (uint32_t)(ks >> 2), jj = (uint32_t)(ks & 3);
                        mma_f16(tmem, sdesc(ab + blk * kRows * 128 + 32 * jj), sdesc(wb + blk * W * 128 + 32 * jj), id_w,
                                ks > 0 ? 1u : 0u);
                    }
                    mma_commit(smem_u32(&bars[0]));
                }
                // layer 0: dX_0 = dY_0 W_0 in column chunks (B = rows c0.. of W_0^T)
                for (int c = 0; c < n_chunks && ok; c++) {
                    if (!mbar_wait(smem_u32(&bars[1]), act_par, abort_flag, status, wlim)) { ok = false; break; }
                    act_par ^= 1u;
                    tc_fence_after();
                    const int c0 = c * (int)kCols;
                    const int nc = in_dim - c0 < (int)kCols ? in_dim - c0 : (int)kCols;
                    const uint32_t wb = smem_u32(sm + lay.wt0_off) + (uint32_t)c0 * 128;
                    for (int ks = 0; ks < lay.ksw; ks++) {
                        uint32_t blk = (uint32_t)(ks >> 2), jj = (uint32_t)(ks & 3);
                        mma_f16(tmem, sdesc(ab + blk * kRows * 128 + 32 * jj),
                                sdesc(wb + blk * (uint32_t)in_dim * 128 + 32 * jj), idesc_f16(fmt, nc), ks > 0 ? 1u : 0u);
                    }
                    mma_commit(smem_u32(&bars[0]));
                }
            }
            mma_commit(smem_u32(&bars[2]));
            volatile int dummy = 0;
            mbar_wait(smem_u32(&bars[2]), 0, &dummy, status);
        }
    } else if (warp >= 2) {
        const int qw = warp & 3;
        const int row = qw * 32 + lane;
        const uint32_t lane_base = tmem + ((uint32_t)(qw * 32) << 16);
        uint8_t* A = sm + lay.a_off;
        uint32_t acc_par = 0;
        bool ok = true;
        auto wait_acc = [&]() -> bool {
            int got = 0;
            if (lane == 0) got = mbar_wait(smem_u32(&bars[0]), acc_par, abort_flag, status, wlim) ? 1 : 0;
            got = __shfl_sync(0xffffffffu, got, 0);
            acc_par ^= 1u;
            if (got) tc_fence_after();
            return got != 0;
        };
        for (int64_t t = blockIdx.x; t < n_tiles && ok; t += gridDim.x) {
            const int64_t grow = t * kRows + row;
            const bool live = grow < n;
            // dY_H = S * dL/dout (16 wide)
            {
                float g[16];
                const float4* src = reinterpret_cast<const float4*>(dout + grow * NIF_OUT);
#pragma unroll
                for (int q = 0; q < 4; q++) {
                    float4 v = live ? src[q] : make_float4(0.f, 0.f, 0.f, 0.f);
                    g[4 * q] = v.x * S; g[4 * q + 1] = v.y * S; g[4 * q + 2] = v.z * S; g[4 * q + 3] = v.w * S;
                }
                uint16_t* drow = live ? dys + ((int64_t)H * n_pad + grow) * ld : nullptr;
#pragma unroll
                for (int c = 0; c < 16; c += 8) {
                    uint4 pk;
                    pk.x = pack2(g[c], g[c + 1], fmt);
                    pk.y = pack2(g[c + 2], g[c + 3], fmt);
                    pk.z = pack2(g[c + 4], g[c + 5], fmt);
                    pk.w = pack2(g[c + 6], g[c + 7], fmt);
                    *reinterpret_cast<uint4*>(A + swz_off(row, c, kRows)) = pk;
                    if (drow) *reinterpret_cast<uint4*>(drow + c) = pk;
                }
                fence_async_smem();
                tc_fence_before();
                mbar_arrive(smem_u32(&bars[1]));
            }
            // layers H .. 1: TMEM holds dX_l; mask with act_{l-1} > 0 -> dY_{l-1}
            for (int l = H; l >= 1; l--) {
                // the activation row for the mask is loaded before waiting on
                // the accumulator, so its latency overlaps the MMAs
                const uint16_t* arow = live ? acts + ((int64_t)(l - 1) * n_pad + grow) * ld : nullptr;
                uint4 am[W / 8];
#pragma unroll
                for (int k = 0; k < W / 8; k++)
                    am[k] = arow ? *reinterpret_cast<const uint4*>(arow + 8 * k) : make_uint4(0, 0, 0, 0);
                if (!wait_acc()) { ok = false; break; }
                uint16_t* drow = live ? dys + ((int64_t)(l - 1) * n_pad + grow) * ld : nullptr;
#pragma unroll
                for (int c0 = 0; c0 < W; c0 += 32) {
                    float v[32];
                    tmem_ld32(lane_base + (uint32_t)c0, v);
#pragma unroll
                    for (int c = 0; c < 32; c += 8) {
                        const uint16_t* a16 = reinterpret_cast<const uint16_t*>(&am[(c0 + c) / 8]);
                        float m[8];
#pragma unroll
                        for (int k = 0; k < 8; k++) m[k] = unpack16(a16[k], fmt) > 0.f ? v[c + k] : 0.f;
                        uint4 pk;
                        pk.x = pack2(m[0], m[1], fmt);
                        pk.y = pack2(m[2], m[3], fmt);
                        pk.z = pack2(m[4], m[5], fmt);
                        pk.w = pack2(m[6], m[7], fmt);
                        *reinterpret_cast<uint4*>(A + swz_off(row, c0 + c, kRows)) = pk;
                        if (drow) *reinterpret_cast<uint4*>(drow + c0 + c) = pk;
                    }
                }
                fence_async_smem();
                tc_fence_before();
                mbar_arrive(smem_u32(&bars[1]));
            }
            // dX_0 chunks -> FP32 rows of dx: each 32 x 32 block of the warp's
            // rows goes through a shared-memory tile so that a store
            // instruction writes 4 rows x 128 contiguous bytes
            float* stg = reinterpret_cast<float*>(sm + lay.st_off) + qw * 32 * kStg;
            for (int c = 0; c < n_chunks && ok; c++) {
                if (!wait_acc()) { ok = false; break; }
                const int c0 = c * (int)kCols;
                const int nc = in_dim - c0 < (int)kCols ? in_dim - c0 : (int)kCols;
                for (int p = 0; p < nc; p += 32) {
                    float v[32];
                    tmem_ld32(lane_base + (uint32_t)p, v);
#pragma unroll
                    for (int k = 0; k < 32; k += 4)
                        *reinterpret_cast<float4*>(stg + lane * kStg + k) = make_float4(v[k], v[k + 1], v[k + 2], v[k + 3]);
                    __syncwarp();
                    const int col4 = (lane & 7) * 4;
#pragma unroll
                    for (int q = 0; q < 8; q++) {
                        const int r = q * 4 + (lane >> 3);
                        const int64_t gr = t * kRows + qw * 32 + r;
                        if (gr < n && col4 < nc - p)
                            *reinterpret_cast<float4*>(dx + gr * in_dim + c0 + p + col4) =
                                *reinterpret_cast<const float4*>(stg + r * kStg + col4);
                    }
                    __syncwarp();
                }
                if (c + 1 < n_chunks) {
                    tc_fence_before();
                    mbar_arrive(smem_u32(&bars[1]));
                }
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kCols) : "memory");
    }
}

// ---------------------------------------------------------------------------
// Weight gradients on tensor cores: dW_l = dY_l^T X_l summed over the rows r,
// computed transposed, D = dW_l^T [in_l x out_l] = X_l^T dY_l, so that both
// operands are the row-major [rows][cols] matrices read as they lie: with
// the rows r as the reduction (K) dimension they are MN-major, and a TMA box
// of 64 columns x 128 rows with 128-byte swizzle is exactly the canonical
// MN-major atom sequence (64 elements x 8 K-rows per 1024-byte atom; the
// next 8 rows 1024 bytes on, the next 64 columns one box (16 KB) on).
// A job is one (layer, 128-column tile of X_l); blockIdx.y splits the row
// chunks. Each CTA keeps its FP32 tile in TMEM over all its chunks and adds
// it to the gradient buffer at the end (one atomic per element and CTA).
// Threads: warp 0 lane 0 TMA, warp 1 lane 0 MMA, all 4 warps the epilogue.
// ---------------------------------------------------------------------------
constexpr int kDwThreads = 128;
constexpr int kDwStages = 4;
constexpr uint32_t kDwBox = 128 * 128;                 // 64 columns x 128 rows of 16-bit
constexpr uint32_t kDwStage = 3 * kDwBox;              // A: 2 boxes, B: 1 box
// unused room after the last stage: an operand read from the last stage with
// its leading and stride offsets taken either way round still ends inside the
// allocation
constexpr uint32_t kDwSlack = 24 * 1024;

struct DwJobs {
    int n;
    int layer[48];
    int i0[48];
    int boxes[48];    // A boxes actually inside X_l's columns (1 or 2)
    int64_t goff[NIF_MAX_LAYERS];   // gradient offset of each layer's [out_l][in_l] block
    int in[NIF_MAX_LAYERS], out[NIF_MAX_LAYERS];
};

__device__ __forceinline__ uint64_t sdesc_mn(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
    d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;     // next 64-element group along M (or N)
    d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;     // next 8 K-rows
    d |= (uint64_t)1 << 46;
    d |= (uint64_t)2 << 61;
    return d;
}

// kind::f16 instruction descriptor with both operands MN-major (bits 15, 16)
__device__ __forceinline__ uint32_t idesc_f16_mn(int fmt, int N) {
    return idesc_f16(fmt, N) | (1u << 15) | (1u << 16);
}

__global__ void __launch_bounds__(kDwThreads, 1)
    k_mlp_dw_tc(const __grid_constant__ CUtensorMap xmap, const __grid_constant__ CUtensorMap amap,
                const __grid_constant__ CUtensorMap dmap, DwJobs jobs, int fmt, int64_t n_max, int64_t n_pad,
                const uint32_t* __restrict__ n_dev, float* __restrict__ grad, int64_t part_stride,
                int* __restrict__ status) {
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    const uint64_t wlim = wait_limit(status);   // bound of the work loop's waits
    uint8_t* sm = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    uint64_t* bars = reinterpret_cast<uint64_t*>(sm + kDwStages * kDwStage + kDwSlack);
    // bars: [0,S) full, [S,2S) empty, 2S acc_full
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 2 * kDwStages + 1);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(bars + 2 * kDwStages + 2);
    const int job = blockIdx.x;
    const int l = jobs.layer[job], i0 = jobs.i0[job], nbox = jobs.boxes[job];
    const int in_l = jobs.in[l], out_l = jobs.out[l];
    const int64_t n = n_dev ? ((int64_t)*n_dev < n_max ? (int64_t)*n_dev : n_max) : n_max;
    const int64_t n_chunks = (n + 127) / 128;
    const int64_t my = (int64_t)blockIdx.y < n_chunks ? (n_chunks - blockIdx.y + gridDim.y - 1) / gridDim.y : 0;
    if (my == 0) return;                          // nothing to add: leave before any setup
    constexpr uint32_t kCols = 64;
    if (tid == 0) {
        for (int i = 0; i < kDwStages; i++) {
            mbar_init(smem_u32(&bars[i]), 1);
            mbar_init(smem_u32(&bars[kDwStages + i]), 1);
        }
        mbar_init(smem_u32(&bars[2 * kDwStages]), 1);
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(kCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;
    const CUtensorMap* am = l == 0 ? &xmap : &amap;
    // row coordinates: X_0 rows r; act_{l-1} rows (l-1) n_pad + r; dY_l rows l n_pad + r
    const int64_t a_row0 = l == 0 ? 0 : (int64_t)(l - 1) * n_pad;
    const int64_t d_row0 = (int64_t)l * n_pad;
    bool ok = true;
    if (warp == 0) {
        if (lane == 0 && my > 0) {
            int slot = 0;
            uint32_t phase = 0, issued_mask = 0, issued_par = 0;
            const uint32_t bytes = (uint32_t)(nbox + 1) * kDwBox;
            for (int64_t j = 0; j < my; j++) {
                const int64_t c = blockIdx.y + j * gridDim.y;
                if (!mbar_wait(smem_u32(&bars[kDwStages + slot]), phase ^ 1u, abort_flag, status, wlim)) { ok = false; break; }
                const uint32_t fb = smem_u32(&bars[slot]);
                const uint32_t st = smem_u32(sm + (uint32_t)slot * kDwStage);
                mbar_expect_tx(fb, bytes);
                for (int b = 0; b < nbox; b++)
                    tma_load_2d(st + (uint32_t)b * kDwBox, am, i0 + 64 * b, (int)(a_row0 + c * 128), fb);
                tma_load_2d(st + 2 * kDwBox, &dmap, 0, (int)(d_row0 + c * 128), fb);
                issued_mask |= 1u << slot;
                issued_par = (issued_par & ~(1u << slot)) | (phase << slot);
                if (++slot == kDwStages) { slot = 0; phase ^= 1u; }
            }
            if (!ok)
                for (int i = 0; i < kDwStages; i++)
                    if (issued_mask >> i & 1u) {
                        volatile int dummy = 0;
                        mbar_wait(smem_u32(&bars[i]), (issued_par >> i) & 1u, &dummy, status);
                    }
        }
    } else if (warp == 1) {
        if (lane == 0 && my > 0) {
            const uint32_t idesc = idesc_f16_mn(fmt, out_l);
            int slot = 0;
            uint32_t phase = 0;
            for (int64_t j = 0; j < my; j++) {
                if (!mbar_wait(smem_u32(&bars[slot]), phase, abort_flag, status, wlim)) { ok = false; break; }
                tc_fence_after();
                const uint32_t st = smem_u32(sm + (uint32_t)slot * kDwStage);
#pragma unroll
                for (int ks = 0; ks < 8; ks++)      // 16 rows per MMA
                    mma_f16(tmem, sdesc_mn(st + 2048u * ks, kDwBox, 1024), sdesc_mn(st + 2 * kDwBox + 2048u * ks, kDwBox, 1024),
                            idesc, (j > 0 || ks > 0) ? 1u : 0u);
                mma_commit(smem_u32(&bars[kDwStages + slot]));
                if (++slot == kDwStages) { slot = 0; phase ^= 1u; }
            }
            mma_commit(smem_u32(&bars[2 * kDwStages]));
            volatile int dummy = 0;
            mbar_wait(smem_u32(&bars[2 * kDwStages]), 0, &dummy, status);
        }
    }
    __syncwarp();
    // epilogue: lane i of the tile holds D[i][0..out_l) = dW_l[0..out_l)[i0 + i]
    if (my > 0) {
        int got = 0;
        if (lane == 0) got = mbar_wait(smem_u32(&bars[2 * kDwStages]), 0, abort_flag, status, wlim) ? 1 : 0;
        got = __shfl_sync(0xffffffffu, got, 0);
        if (got && !*abort_flag) {
            tc_fence_after();
            const int i = i0 + warp * 32 + lane;
            const uint32_t lane_base = tmem + ((uint32_t)(warp * 32) << 16);
            // part_stride > 0 (deterministic mode): grad holds one copy of the
            // weight blocks per row range, each range's sum is stored in its own
            float* g = grad + (int64_t)blockIdx.y * part_stride + jobs.goff[l] + i;
            for (int c0 = 0; c0 < out_l; c0 += 16) {
                float v[16];
                tmem_ld16(lane_base + (uint32_t)c0, v);
                if (i < in_l) {
                    if (part_stride > 0) {
#pragma unroll
                        for (int k = 0; k < 16; k++) g[(int64_t)(c0 + k) * in_l] = v[k];
                    } else {
#pragma unroll
                        for (int k = 0; k < 16; k++) atomicAdd(g + (int64_t)(c0 + k) * in_l, v[k]);
                    }
                }
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kCols) : "memory");
    }
}

// rows [n, min(roundup(n, 128), n_max)) of x and [n, roundup(n, 128)) of every
// stacked activation / dY layer are zeroed so that the weight-gradient MMAs
// read finite zeros past the last live row
__global__ void k_zero_tail(const uint32_t* __restrict__ n_dev, int64_t n_max, int64_t n_pad, uint16_t* x, int in_dim,
                            uint16_t* acts, int n_acts, uint16_t* dys, int n_dys, int ld) {
    const int64_t n = n_dev ? ((int64_t)*n_dev < n_max ? (int64_t)*n_dev : n_max) : n_max;
    const int64_t end = (n + 127) / 128 * 128;
    const int64_t rows = end - n;
    if (rows <= 0) return;
    const int64_t xr = (end < n_max ? end : n_max) - n;
    const int64_t tot_x = x ? (xr > 0 ? xr : 0) * in_dim : 0;
    const int64_t per = rows * ld;
    const int64_t tot = tot_x + (int64_t)(n_acts + n_dys) * per;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < tot; e += (int64_t)gridDim.x * blockDim.x) {
        if (e < tot_x) {
            x[n * in_dim + e] = 0;
            continue;
        }
        int64_t f = e - tot_x;
        int layer = (int)(f / per);
        int64_t r = f % per;
        if (layer < n_acts) acts[((int64_t)layer * n_pad + n) * ld + r] = 0;
        else dys[((int64_t)(layer - n_acts) * n_pad + n) * ld + r] = 0;
    }
}

}  // namespace

PFN_cuTensorMapEncodeTiled_v12000 g_encode_tiled = nullptr;

nif_status get_encoder(nif_handle* h) {
    if (g_encode_tiled) return NIF_OK;
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q);
    if (e != cudaSuccess || q != cudaDriverEntryPointSuccess || !fn)
        return nif_fail(h, NIF_ERR_CUDA, "cuTensorMapEncodeTiled unavailable");
    g_encode_tiled = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
    return NIF_OK;
}

namespace {

TcLayout make_layout(int W, int K0, int H) {
    TcLayout L{};
    L.nb0 = (K0 + 63) / 64;
    L.ks0 = (K0 + 15) / 16;
    L.nbw = (W + 63) / 64;
    L.ksw = W / 16;
    uint32_t off = 0;
    L.wo_off = 0;
    off += (uint32_t)L.nbw * 16 * 128;
    L.w0_off = off;
    off += (uint32_t)L.nb0 * W * 128;
    L.wh_off = off;
    off += (uint32_t)(H - 1) * L.nbw * W * 128;
    L.a_off = off;
    off += 2u * (uint32_t)L.nbw * kRows * 128;      // one activation tile per accumulator stage
    L.x_off = off;
    // ring depth from what is left of the shared memory budget
    const uint32_t budget = 220 * 1024;
    int S = (int)((budget - off - 1024 - 256) / kStageBytes);
    if (S > 12) S = 12;
    L.stages = S;
    off += (uint32_t)S * kStageBytes;
    L.bar_off = off;
    off += 8 * (2 * S + 6) + 16;
    L.total = off + 1024;        // room to align the dynamic buffer to 1024 bytes
    return L;
}

template <int W>
nif_status launch_tc(nif_handle* h, const void* x, int dtype, int64_t n, const uint32_t* n_dev, float* out,
                     uint16_t* acts_out, int64_t acts_rows, int acts_ld, cudaStream_t s, int ctas) {
    TcLayout lay = make_layout(W, h->in_dim, h->H);
    for (int l = 0; l < h->n_layers; l++) {
        lay.woff[l] = (uint32_t)(h->off_layer[l] - h->off_layer[0]);
        if (lay.woff[l] % 8) return nif_fail(h, NIF_ERR_STATE, "weight copy not 16-byte aligned per layer");
    }
    if (lay.stages < 2) return nif_fail(h, NIF_ERR_ARG, "tensor-core MLP: weights do not fit in shared memory");
    CUtensorMap map;
    cuuint64_t gdim[2] = {(cuuint64_t)h->in_dim, (cuuint64_t)n};
    cuuint64_t gstride[1] = {(cuuint64_t)h->in_dim * 2};
    cuuint32_t box[2] = {64, kRows};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = g_encode_tiled(&map, dtype == NIF_BF16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT16,
                                2, const_cast<void*>(x), gdim, gstride, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                                CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                                CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return nif_fail(h, NIF_ERR_ARG, "cuTensorMapEncodeTiled failed for the feature matrix");
    NIF_CK(h, cudaFuncSetAttribute(k_mlp_tc<W>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)lay.total));
    int64_t n_tiles = (n + kRows - 1) / kRows;
    int grid = (int)std::min<int64_t>(n_tiles, ctas > 0 ? std::min(ctas, h->num_sms) : h->num_sms);
    const uint16_t* w = reinterpret_cast<const uint16_t*>(dtype == NIF_BF16 ? (const void*)h->d_w_bf16
                                                                             : (const void*)h->d_w_f16);
    k_mlp_tc<W><<<grid, kThreads, lay.total, s>>>(map, lay, w, h->in_dim, h->H, dtype == NIF_BF16 ? 1 : 0, n, n_dev,
                                                  out, acts_out, acts_rows, acts_ld, h->d_status);
    NIF_CK_LAUNCH(h);
    return NIF_OK;
}

}  // namespace

nif_status nif_mlp_fwd_tc_run(nif_handle* h, const void* x, int dtype, const uint32_t* n_dev, int64_t n_max,
                              float* out, cudaStream_t s) {
    return nif_mlp_fwd_tc_acts_run(h, x, dtype, n_dev, n_max, out, nullptr, 0, 0, s);
}

nif_status nif_mlp_fwd_tc_acts_run(nif_handle* h, const void* x, int dtype, const uint32_t* n_dev, int64_t n_max,
                                   float* out, uint16_t* acts_out, int64_t acts_rows, int acts_ld, cudaStream_t s,
                                   int ctas) {
    NifProf prof_(h, "mlp_fwd_tc", s);
    if (n_max <= 0) return NIF_OK;
    if (dtype != NIF_BF16 && dtype != NIF_FP16) return nif_fail(h, NIF_ERR_ARG, "tensor-core MLP dtype");
    if (h->in_dim % 8 != 0) return nif_fail(h, NIF_ERR_ARG, "tensor-core MLP needs in_dim % 8 == 0");
    if ((reinterpret_cast<uintptr_t>(x) & 15) != 0) return nif_fail(h, NIF_ERR_ARG, "feature matrix not 16-byte aligned");
    nif_status st = get_encoder(h);
    if (st != NIF_OK) return st;
    if ((st = nif_refresh_lowp(h, s)) != NIF_OK) return st;
    switch (h->W) {
        case 32: return launch_tc<32>(h, x, dtype, n_max, n_dev, out, acts_out, acts_rows, acts_ld, s, ctas);
        case 64: return launch_tc<64>(h, x, dtype, n_max, n_dev, out, acts_out, acts_rows, acts_ld, s, ctas);
        case 128: return launch_tc<128>(h, x, dtype, n_max, n_dev, out, acts_out, acts_rows, acts_ld, s, ctas);
        default: return nif_fail(h, NIF_ERR_ARG, "tensor-core MLP width must be 32, 64 or 128");
    }
}

namespace {

template <int W>
static nif_status launch_tc_bwd(nif_handle* h, const float* dout, const uint16_t* acts, const uint32_t* n_dev,
                                int64_t n_max, int64_t n_pad, int ld, uint16_t* dys, float* dx, cudaStream_t s) {
    TcBwdLayout lay{};
    lay.nbw = (W + 63) / 64;
    lay.ksw = W / 16;
    uint32_t off = 0;
    lay.wto_off = off;
    off += (uint32_t)W * 128;
    lay.wth_off = off;
    off += (uint32_t)(h->H - 1) * lay.nbw * W * 128;
    lay.wt0_off = off;
    off += (uint32_t)lay.nbw * h->in_dim * 128;
    off = (off + 1023) & ~1023u;
    lay.a_off = off;
    off += (uint32_t)lay.nbw * kRows * 128;
    lay.st_off = off;
    off += 4u * 32u * kStg * 4u;
    lay.bar_off = off;
    off += 64;
    lay.total = off + 1024;
    if (lay.total > 227 * 1024)
        return nif_fail(h, NIF_ERR_ARG, "tensor-core backward: transposed weights do not fit in shared memory");
    for (int l = 0; l < h->n_layers; l++) lay.wtoff[l] = (uint32_t)(h->off_layer[l] - h->off_layer[0]);
    NIF_CK(h, cudaFuncSetAttribute(k_mlp_tc_bwd<W>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)lay.total));
    int64_t n_tiles = (n_max + kRows - 1) / kRows;
    int grid = (int)std::min<int64_t>(n_tiles, h->num_sms);
    const int fmt = h->cfg.precision == NIF_BF16 ? 1 : 0;
    const uint16_t* wt = reinterpret_cast<const uint16_t*>(fmt ? (const void*)h->d_wt_bf16 : (const void*)h->d_wt_f16);
    k_mlp_tc_bwd<W><<<grid, kThreads, lay.total, s>>>(lay, wt, h->in_dim, h->H, fmt, n_max, n_pad, ld, n_dev, dout,
                                                     acts, &h->d_ls->scale, dys, dx, h->d_status);
    NIF_CK_LAUNCH(h);
    return NIF_OK;
}

static nif_status map_2d(nif_handle* h, CUtensorMap* map, const void* base, int dtype, uint64_t inner, uint64_t outer,
                         uint64_t row_elems, const char* what) {
    cuuint64_t gdim[2] = {(cuuint64_t)inner, (cuuint64_t)outer};
    cuuint64_t gstride[1] = {(cuuint64_t)row_elems * 2};
    cuuint32_t box[2] = {64, kRows};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = g_encode_tiled(map, dtype == NIF_BF16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT16,
                                2, const_cast<void*>(base), gdim, gstride, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                                CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                                CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return nif_fail(h, NIF_ERR_ARG, std::string("cuTensorMapEncodeTiled failed for ") + what);
    return NIF_OK;
}

}  // namespace

nif_status nif_mlp_bwd_tc_run(nif_handle* h, const float* dout, const uint16_t* acts, const uint32_t* n_dev,
                              int64_t n_max, int64_t n_pad, int ld, uint16_t* dys, float* dx, cudaStream_t s) {
    NifProf prof_(h, "mlp_bwd_tc", s);
    if (n_max <= 0) return NIF_OK;
    if (h->in_dim % 16 != 0) return nif_fail(h, NIF_ERR_ARG, "tensor-core backward needs in_dim % 16 == 0");
    if (h->cfg.precision != NIF_BF16 && h->cfg.precision != NIF_FP16)
        return nif_fail(h, NIF_ERR_ARG, "tensor-core backward needs a BF16 or FP16 handle");
    nif_status st = nif_refresh_lowp(h, s);
    if (st != NIF_OK) return st;
    switch (h->W) {
        case 32: return launch_tc_bwd<32>(h, dout, acts, n_dev, n_max, n_pad, ld, dys, dx, s);
        case 64: return launch_tc_bwd<64>(h, dout, acts, n_dev, n_max, n_pad, ld, dys, dx, s);
        default: return nif_fail(h, NIF_ERR_ARG, "tensor-core backward width must be 32 or 64");
    }
}

nif_status nif_mlp_dw_tc_run(nif_handle* h, const void* x16, const uint16_t* acts, const uint16_t* dys,
                             const uint32_t* n_dev, int64_t n_max, int64_t n_pad, int ld, cudaStream_t s) {
    NifProf prof_(h, "mlp_dw_tc", s);
    if (n_max <= 0) return NIF_OK;
    if (h->W > 64 || ld != 64) return nif_fail(h, NIF_ERR_ARG, "tensor-core weight gradients need W <= 64, ld 64");
    const int dtype = h->cfg.precision;
    nif_status st = get_encoder(h);
    if (st != NIF_OK) return st;
    CUtensorMap xm, am, dm;
    if ((st = map_2d(h, &xm, x16, dtype, h->in_dim, n_max, h->in_dim, "the feature matrix")) != NIF_OK) return st;
    if ((st = map_2d(h, &am, acts, dtype, ld, (uint64_t)h->H * n_pad, ld, "the activations")) != NIF_OK) return st;
    if ((st = map_2d(h, &dm, dys, dtype, ld, (uint64_t)(h->H + 1) * n_pad, ld, "the output gradients")) != NIF_OK)
        return st;
    // zero the rows past the live count in the last 128-row chunk
    k_zero_tail<<<h->num_sms, 256, 0, s>>>(n_dev, n_max, n_pad, n_dev ? (uint16_t*)x16 : nullptr, h->in_dim,
                                           (uint16_t*)acts, h->H, (uint16_t*)dys, h->H + 1, ld);
    NIF_CK_LAUNCH(h);
    DwJobs jobs{};
    // deterministic mode: offsets within the weights' span [off_layer[0], wend)
    const int64_t wbase = h->det ? (int64_t)h->off_layer[0] : 0;
    const int64_t wcnt = (int64_t)h->off_layer[h->n_layers - 1] +
                         (int64_t)h->lay_out[h->n_layers - 1] * h->lay_in[h->n_layers - 1] - (int64_t)h->off_layer[0];
    for (int l = 0; l < h->n_layers; l++) {
        const int in_l = h->lay_in[l];
        jobs.goff[l] = (int64_t)h->off_layer[l] - wbase;
        jobs.in[l] = in_l;
        jobs.out[l] = h->lay_out[l];
        for (int i0 = 0; i0 < in_l; i0 += 128) {
            if (jobs.n >= 48) return nif_fail(h, NIF_ERR_ARG, "too many weight-gradient tiles");
            jobs.layer[jobs.n] = l;
            jobs.i0[jobs.n] = i0;
            jobs.boxes[jobs.n] = in_l - i0 > 64 ? 2 : 1;
            jobs.n++;
        }
    }
    const uint32_t smem = kDwStages * kDwStage + kDwSlack + 8 * (2 * kDwStages + 4) + 1024;
    NIF_CK(h, cudaFuncSetAttribute(k_mlp_dw_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    const int64_t chunks = (n_max + 127) / 128;
    int splits = (int)std::max<int64_t>(1, std::min<int64_t>(chunks, (h->num_sms + jobs.n - 1) / jobs.n));
    dim3 grid(jobs.n, splits);
    float* part = nullptr;
    if (h->det) {
        // each row range's sums kept apart (a range with no live rows leaves zeros)
        if ((st = nif_grow(h, h->b_parts, sizeof(float) * (size_t)splits * wcnt)) != NIF_OK) return st;
        part = (float*)h->b_parts.p;
        NIF_CK(h, cudaMemsetAsync(part, 0, sizeof(float) * (size_t)splits * wcnt, s));
    }
    k_mlp_dw_tc<<<grid, kDwThreads, smem, s>>>(xm, am, dm, jobs, dtype == NIF_BF16 ? 1 : 0, n_max, n_pad, n_dev,
                                               part ? part : h->d_grad, part ? wcnt : 0, h->d_status);
    NIF_CK_LAUNCH(h);
    if (part) return nif_sum_parts_run(h, part, splits, wcnt, h->d_grad + wbase, s);
    return NIF_OK;
}
