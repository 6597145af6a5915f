// k_mlp_x3.cu -- the FP32 path of the MLP (Sec. 2, Fig. 2d: H hidden ReLU
// layers without bias and a linear output layer), forward and backward, on
// the tcgen05 tensor cores at FP32 accuracy by split TF32.
//
// Every FP32 operand x is split as x = hi + lo, hi = x rounded to TF32 (10
// fraction bits) and lo = x - hi (exact in FP32). A product a*b is taken as
// hi_a hi_b + hi_a lo_b + lo_a hi_b: three kind::tf32 MMAs into the same
// FP32 accumulator in TMEM. The dropped lo_a lo_b is below 2^-22 |ab| and lo
// enters the MMA with 10 fraction bits, so a product carries a relative
// error of about 2^-21 (one plain TF32 product: 2^-11); sums accumulate in
// FP32 as in the FFMA path.
//
// k_gemm_x3: C = epi(A B^T) with A [rows x K] row-major FP32 (features,
//   activations or output gradients, read by TMA as they lie: the rows are
//   M, K is contiguous) and B [N x K] a weight matrix or its transpose,
//   whose hi and lo copies are written once per parameter update. One
//   persistent CTA per SM walks jobs (128-row tile, chunk of <= 256 of the
//   N columns). Warp roles:
//     warp 0     TMA: per 32-deep k-block the A box (128 rows x 32 FP32,
//                128-byte swizzle) and the hi and lo boxes of B;
//     warps 6-9  split the A box in place into hi and a lo copy;
//     warp 1     issues the k-block's 12 MMAs (4 k-steps x 3 products) into
//                one of two TMEM accumulators, so the epilogue of one job
//                overlaps the MMAs of the next;
//     warps 2-5  epilogue: TMEM -> registers -> ReLU or ReLU-derivative
//                mask -> per-warp shared-memory transpose -> 128-byte
//                coalesced stores of the live rows only.
//   The ReLU-derivative mask (the layer's stored activations) of a job is
//   loaded by TMA into one of two shared-memory buffers, one per TMEM
//   accumulator, when the producer starts the job, so the epilogue never
//   waits on global loads.
// k_dw_x3: weight gradient dW_l^T = X_l^T dY_l summed over the rows. The
//   rows are the reduction (K) dimension, so the converter warps transpose
//   the row-major boxes of X_l and dY_l (TMA, no swizzle) into K-major
//   operands while they split them; each CTA keeps its [128 x out_l] tile in
//   TMEM over its share of the rows and adds it to the gradient once.
// Every wait on an mbarrier is bounded in time; on expiry the kernel records
// NIF_ERR_TIMEOUT, drains its own copies and MMAs, frees TMEM and returns.
#include <algorithm>

#include "nif_internal.cuh"
#include "tc_ptx.cuh"

namespace {

constexpr int kX3Threads = 320;               // 10 warps
constexpr uint32_t kABox = 128u * 128u;       // 128 rows x 32 FP32 = 16 KB
constexpr uint32_t kX3Budget = 220u * 1024u;  // dynamic shared memory a CTA may use

__device__ __forceinline__ void split_tf32(float x, float& hi, float& lo) {
    // round to nearest (ties away from zero) at 10 fraction bits, then the exact remainder
    hi = __uint_as_float((__float_as_uint(x) + 0x1000u) & 0xFFFFE000u);
    lo = x - hi;
}

__device__ __forceinline__ void split4(float4 v, float4& h, float4& l) {
    split_tf32(v.x, h.x, l.x);
    split_tf32(v.y, h.y, l.y);
    split_tf32(v.z, h.z, l.z);
    split_tf32(v.w, h.w, l.w);
}

// kind::tf32 instruction descriptor: FP32 accumulator (bit 4), A and B TF32
// (format 2 at bits 7 and 10), both K-major, N >> 3 at bit 17, M = 128.
__device__ __forceinline__ uint32_t idesc_tf32(int N) {
    return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
}

__device__ __forceinline__ void mma_tf32(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accum) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accum)
        : "memory");
}

// The three products of one 8-deep k-step at byte offset `o` of the operands.
__device__ __forceinline__ void mma_x3(uint32_t acc, uint32_t ah, uint32_t al, uint32_t bh, uint32_t bl, uint32_t o,
                                       uint32_t idesc, uint32_t accum) {
    mma_tf32(acc, sdesc(ah + o), sdesc(bh + o), idesc, accum);
    mma_tf32(acc, sdesc(ah + o), sdesc(bl + o), idesc, 1u);
    mma_tf32(acc, sdesc(al + o), sdesc(bh + o), idesc, 1u);
}

enum X3Epi { kX3Store = 0, kX3Relu = 1, kX3Mask = 2 };

struct X3Args {
    float* C; int64_t ldc;            // C(r, j) = C[r * ldc + j], j < N
    const float* mask; int64_t ldm;   // kX3Mask: C(r, j) kept where mask[r * ldm + j] > 0
    int N, NB, n_chunks;              // columns, columns per job, jobs per row tile
    int nkb;                          // 32-deep k-blocks
    int stages;
    uint32_t stage_bytes, b_bytes;    // one stage; one B box (NB rows x 128 bytes)
    uint32_t stg_off, bar_off;
    uint32_t msk_off, msk_bytes;      // kX3Mask: two mask tiles (128 rows x NB FP32, boxes of mbox columns)
    int mbox;
    uint32_t acc_stride, tmem_cols;   // TMEM columns per accumulator and in all
    int64_t n_max;                    // rows of A and C
    int b_lo_row;                     // first row of B's lo copy in the stacked [hi; lo] matrix
};

// Stage `CNT` accumulator columns of this warp's 32 rows through shared memory
// and store the live rows with 16-byte vectors, a row's CNT*4 bytes contiguous.
// msk: this warp's first row in the job's mask tile, at this chunk's column box
template <int EPI, int CNT>
__device__ __forceinline__ void x3_store(const X3Args& a, uint8_t* stg, const float* v, const float* msk, int lane,
                                         int64_t row0, int64_t n, int col0) {
    constexpr int CPR = CNT / 4;     // 16-byte chunks per row
    constexpr int RPP = 32 / CPR;    // rows per pass
#pragma unroll
    for (int ch = 0; ch < CPR; ch++)
        *reinterpret_cast<float4*>(stg + lane * 128 + ((ch ^ (lane & 7)) << 4)) =
            make_float4(v[4 * ch], v[4 * ch + 1], v[4 * ch + 2], v[4 * ch + 3]);
    __syncwarp();
#pragma unroll
    for (int p = 0; p < CPR; p++) {
        const int r = p * RPP + lane / CPR, ch = lane % CPR;
        const int64_t g = row0 + r;
        const int col = col0 + ch * 4;
        float4 w = *reinterpret_cast<const float4*>(stg + r * 128 + ((ch ^ (r & 7)) << 4));
        if (g < n && col < a.N) {
            if (EPI == kX3Mask) {
                const float4 m = *reinterpret_cast<const float4*>(msk + r * a.mbox + ch * 4);
                w.x = m.x > 0.f ? w.x : 0.f;
                w.y = m.y > 0.f ? w.y : 0.f;
                w.z = m.z > 0.f ? w.z : 0.f;
                w.w = m.w > 0.f ? w.w : 0.f;
            }
            *reinterpret_cast<float4*>(a.C + g * a.ldc + col) = w;
        }
    }
    __syncwarp();
}

template <int EPI>
__global__ void __launch_bounds__(kX3Threads, 1)
    k_gemm_x3(const __grid_constant__ CUtensorMap amap, const __grid_constant__ CUtensorMap bmap,
              const __grid_constant__ CUtensorMap mmap, X3Args a, const uint32_t* __restrict__ n_dev,
              int* __restrict__ status) {
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    const uint64_t wlim = wait_limit(status);   // bound of the work loop's waits
    uint8_t* sm = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int S = a.stages;
    uint64_t* bars = reinterpret_cast<uint64_t*>(sm + a.bar_off);
    // [0,S) loaded, [S,2S) split, [2S,3S) free, 3S+{0,1} acc full, 3S+{2,3} acc (and mask tile) free,
    // 3S+4 drain, 3S+{5,6} mask tile loaded
    const int B_CONV = S, B_EMPTY = 2 * S, B_ACC = 3 * S, B_ACCE = 3 * S + 2, B_DRAIN = 3 * S + 4, B_MSK = 3 * S + 5;
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 3 * S + 7);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(bars + 3 * S + 8);
    const int64_t n = n_dev ? ((int64_t)*n_dev < a.n_max ? (int64_t)*n_dev : a.n_max) : a.n_max;
    const int64_t n_jobs = (n + 127) / 128 * a.n_chunks;
    const int64_t my = (int64_t)blockIdx.x < n_jobs ? (n_jobs - blockIdx.x + gridDim.x - 1) / gridDim.x : 0;
    // a CTA without jobs (a chunk whose device count is short or zero) leaves
    // before any barrier, tensor memory or copy: uniform per CTA
    if (my == 0) return;

    if (tid == 0) {
        for (int i = 0; i < S; i++) {
            mbar_init(smem_u32(&bars[i]), 1);
            mbar_init(smem_u32(&bars[B_CONV + i]), 128);
            mbar_init(smem_u32(&bars[B_EMPTY + i]), 1);
        }
        for (int q = 0; q < 2; q++) {
            mbar_init(smem_u32(&bars[B_ACC + q]), 1);
            mbar_init(smem_u32(&bars[B_ACCE + q]), 128);
            mbar_init(smem_u32(&bars[B_MSK + q]), 1);
        }
        mbar_init(smem_u32(&bars[B_DRAIN]), 1);
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(a.tmem_cols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    if (warp == 0) {
        // ---------------- TMA producer ----------------
        if (lane == 0) {
            asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&amap)) : "memory");
            asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&bmap)) : "memory");
            int slot = 0;
            uint32_t phase = 0, issued_mask = 0, issued_par = 0;
            uint32_t mf_issued = 0, mf_par = 0, me_par[2] = {0u, 0u};
            bool ok = true;
            for (int64_t j = 0; j < my && ok; j++) {
                const int64_t job = blockIdx.x + j * gridDim.x;
                const int tile = (int)(job / a.n_chunks), chunk = (int)(job % a.n_chunks);
                if (EPI == kX3Mask) {
                    // the job's mask tile, once the epilogue is done with the buffer's previous job
                    const int q = (int)(j & 1);
                    if (j >= 2) {
                        if (!mbar_wait(smem_u32(&bars[B_ACCE + q]), me_par[q], abort_flag, status, wlim)) { ok = false; break; }
                        me_par[q] ^= 1u;
                    }
                    const uint32_t mb = smem_u32(&bars[B_MSK + q]);
                    const uint32_t dst = smem_u32(sm + a.msk_off + (uint32_t)q * a.msk_bytes);
                    mbar_expect_tx(mb, a.msk_bytes);
                    for (int b = 0; b * a.mbox < a.NB; b++)
                        tma_load_2d(dst + (uint32_t)b * 128u * (uint32_t)a.mbox * 4u, &mmap, chunk * a.NB + b * a.mbox,
                                    tile * 128, mb);
                    mf_issued |= 1u << q;
                    mf_par = (mf_par & ~(1u << q)) | ((uint32_t)((j >> 1) & 1) << q);
                }
                for (int kb = 0; kb < a.nkb; kb++) {
                    if (!mbar_wait(smem_u32(&bars[B_EMPTY + slot]), phase ^ 1u, abort_flag, status, wlim)) { ok = false; break; }
                    const uint32_t fb = smem_u32(&bars[slot]);
                    const uint32_t st = smem_u32(sm + (uint32_t)slot * a.stage_bytes);
                    mbar_expect_tx(fb, kABox + 2u * a.b_bytes);
                    tma_load_2d(st, &amap, kb * 32, tile * 128, fb);
                    tma_load_2d(st + 2u * kABox, &bmap, kb * 32, chunk * a.NB, fb);
                    tma_load_2d(st + 2u * kABox + a.b_bytes, &bmap, kb * 32, a.b_lo_row + chunk * a.NB, fb);
                    issued_mask |= 1u << slot;
                    issued_par = (issued_par & ~(1u << slot)) | (phase << slot);
                    if (++slot == S) { slot = 0; phase ^= 1u; }
                }
            }
            // every issued copy must have landed before the CTA exits
            for (int i = 0; i < S; i++)
                if (issued_mask >> i & 1u) {
                    volatile int dummy = 0;
                    mbar_wait(smem_u32(&bars[i]), (issued_par >> i) & 1u, &dummy, status);
                }
            for (int q = 0; q < 2; q++)
                if (mf_issued >> q & 1u) {
                    volatile int dummy = 0;
                    mbar_wait(smem_u32(&bars[B_MSK + q]), (mf_par >> q) & 1u, &dummy, status);
                }
        }
    } else if (warp == 1) {
        // ---------------- MMA issuer ----------------
        if (lane == 0) {
            const uint32_t idesc = idesc_tf32(a.NB);
            int slot = 0;
            uint32_t phase = 0;
            uint32_t ae_par[2] = {0u, 0u};
            bool ok = true;
            for (int64_t j = 0; j < my && ok; j++) {
                const int q = (int)(j & 1);
                const uint32_t acc = tmem + (uint32_t)q * a.acc_stride;
                if (j >= 2) {   // the epilogue must have read this accumulator out
                    if (!mbar_wait(smem_u32(&bars[B_ACCE + q]), ae_par[q], abort_flag, status, wlim)) { ok = false; break; }
                    ae_par[q] ^= 1u;
                    tc_fence_after();
                }
                for (int kb = 0; kb < a.nkb; kb++) {
                    if (!mbar_wait(smem_u32(&bars[B_CONV + slot]), phase, abort_flag, status, wlim)) { ok = false; break; }
                    tc_fence_after();
                    const uint32_t ah = smem_u32(sm + (uint32_t)slot * a.stage_bytes);
                    const uint32_t al = ah + kABox, bh = ah + 2u * kABox, bl = bh + a.b_bytes;
#pragma unroll
                    for (int ks = 0; ks < 4; ks++)
                        mma_x3(acc, ah, al, bh, bl, 32u * ks, idesc, (kb > 0 || ks > 0) ? 1u : 0u);
                    mma_commit(smem_u32(&bars[B_EMPTY + slot]));   // frees the stage when these MMAs finish
                    if (++slot == S) { slot = 0; phase ^= 1u; }
                }
                if (!ok) break;
                mma_commit(smem_u32(&bars[B_ACC + q]));
            }
            // all MMAs of this CTA complete before TMEM is released
            mma_commit(smem_u32(&bars[B_DRAIN]));
            volatile int dummy = 0;
            mbar_wait(smem_u32(&bars[B_DRAIN]), 0, &dummy, status);
        }
    } else if (warp >= 6) {
        // ---------------- splitter: A box -> hi in place + lo copy ----------------
        const int ct = tid - 192;
        int slot = 0;
        uint32_t phase = 0;
        for (int64_t j = 0; j < my; j++) {
            bool ok = true;
            for (int kb = 0; kb < a.nkb; kb++) {
                if (!mbar_wait(smem_u32(&bars[slot]), phase, abort_flag, status, wlim)) { ok = false; break; }
                float4* A = reinterpret_cast<float4*>(sm + (uint32_t)slot * a.stage_bytes);
                float4* Al = reinterpret_cast<float4*>(sm + (uint32_t)slot * a.stage_bytes + kABox);
#pragma unroll
                for (int i = 0; i < 8; i++) {
                    const int idx = ct + 128 * i;
                    float4 h, l;
                    split4(A[idx], h, l);
                    A[idx] = h;
                    Al[idx] = l;
                }
                fence_async_smem();
                mbar_arrive(smem_u32(&bars[B_CONV + slot]));
                if (++slot == S) { slot = 0; phase ^= 1u; }
            }
            if (!ok) break;
        }
    } else {
        // ---------------- epilogue (warps 2..5) ----------------
        const int qw = warp & 3;                  // TMEM lane quarter this warp may access
        uint8_t* stg = sm + a.stg_off + (uint32_t)(warp - 2) * 4096u;
        uint32_t af_par[2] = {0u, 0u}, mk_par[2] = {0u, 0u};
        for (int64_t j = 0; j < my; j++) {
            const int q = (int)(j & 1);
            const int64_t job = blockIdx.x + j * gridDim.x;
            const int64_t tile = job / a.n_chunks;
            const int chunk = (int)(job % a.n_chunks);
            int got = 0;
            if (lane == 0) got = mbar_wait(smem_u32(&bars[B_ACC + q]), af_par[q], abort_flag, status, wlim) ? 1 : 0;
            got = __shfl_sync(0xffffffffu, got, 0);
            if (!got) break;
            af_par[q] ^= 1u;
            if (EPI == kX3Mask) {
                if (!mbar_wait(smem_u32(&bars[B_MSK + q]), mk_par[q], abort_flag, status, wlim)) break;
                mk_par[q] ^= 1u;
            }
            tc_fence_after();
            const uint32_t tb = tmem + ((uint32_t)(qw * 32) << 16) + (uint32_t)q * a.acc_stride;
            const int64_t row0 = tile * 128 + qw * 32;
            // this warp's rows of the job's mask tile (column boxes of mbox, 128 rows each)
            const float* msk = reinterpret_cast<const float*>(sm + a.msk_off + (uint32_t)q * a.msk_bytes) + qw * 32 * a.mbox;
            for (int c0 = 0; c0 < a.NB; c0 += 32) {
                float v[32];
                const float* mc = msk + (c0 / 32) * 128 * a.mbox;   // mbox is 32 whenever c0 > 0
                if (a.NB - c0 >= 32) {
                    tmem_ld32(tb + (uint32_t)c0, v);
                    if (EPI == kX3Relu)
#pragma unroll
                        for (int i = 0; i < 32; i++) v[i] = fmaxf(v[i], 0.f);
                    x3_store<EPI, 32>(a, stg, v, mc, lane, row0, n, chunk * a.NB + c0);
                } else {
                    tmem_ld16(tb + (uint32_t)c0, v);
                    if (EPI == kX3Relu)
#pragma unroll
                        for (int i = 0; i < 16; i++) v[i] = fmaxf(v[i], 0.f);
                    x3_store<EPI, 16>(a, stg, v, mc, lane, row0, n, chunk * a.NB + c0);
                }
            }
            tc_fence_before();
            mbar_arrive(smem_u32(&bars[B_ACCE + q]));
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(a.tmem_cols) : "memory");
    }
}

// ---------------------------------------------------------------------------
// The whole FP32 forward in one persistent kernel (hidden width W = 32 or 64):
// per 128-row tile, layer 0 streams the input rows through the TMA ring as in
// k_gemm_x3 (A box 128 x 32 FP32 split in place into hi plus a lo copy, with
// the hi and lo boxes of W_0), and layers 1..H read their A operand from a
// shared-memory activation tile that the epilogue writes, split into hi and
// lo in the K-major 128-byte-swizzled layout, right after the ReLU of the
// layer before. The hidden layers' split weights stream through the same
// ring (B boxes only). The epilogue also stores every hidden activation row
// to global memory (the backward needs them) and the 16 outputs of the last
// layer. Two TMEM accumulators: the MMAs of a tile's layer 0 overlap the
// epilogue of the tile before's last layer. Warp roles as k_gemm_x3: 0 TMA,
// 1 MMA issue, 2-5 epilogue, 6-9 splitter.
// ---------------------------------------------------------------------------
struct X3FwdArgs {
    float* acts;                      // [H][n_max][W]
    float* out;                       // [n_max][NIF_OUT]
    int64_t n_max;
    int K0, W, H;                     // input width, hidden width, hidden layers
    int nkb0, nkbw;                   // 32-deep k-blocks of layer 0 and of a W-deep layer
    int stages;
    uint32_t stage_bytes;             // A hi + A lo + B hi + B lo (B boxes W rows)
    uint32_t act_off, stg_off, bar_off;
    uint32_t acc_stride, tmem_cols;
};

struct X3FwdMaps {
    CUtensorMap w[NIF_MAX_LAYERS];    // [hi; lo] copy of layer l's weight, boxes 32 (K) x out_l rows
};

template <int W>
__global__ void __launch_bounds__(kX3Threads, 1)
    k_mlp_x3_fwd(const __grid_constant__ CUtensorMap amap, const __grid_constant__ X3FwdMaps wm, X3FwdArgs a,
                 const uint32_t* __restrict__ n_dev, int* __restrict__ status) {
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    const uint64_t wlim = wait_limit(status);   // bound of the work loop's waits
    uint8_t* sm = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int S = a.stages, H = a.H;
    constexpr int KBW = W / 32;                  // k-blocks of a W-deep layer
    uint64_t* bars = reinterpret_cast<uint64_t*>(sm + a.bar_off);
    // [0,S) loaded, [S,2S) split, [2S,3S) free, 3S+{0,1} acc full, 3S+{2,3} acc free, 3S+4 act tile ready,
    // 3S+5 drain
    const int B_CONV = S, B_EMPTY = 2 * S, B_ACC = 3 * S, B_ACCE = 3 * S + 2, B_ACT = 3 * S + 4, B_DRAIN = 3 * S + 5;
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 3 * S + 6);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(bars + 3 * S + 7);
    const int64_t n = n_dev ? ((int64_t)*n_dev < a.n_max ? (int64_t)*n_dev : a.n_max) : a.n_max;
    const int64_t n_tiles = (n + 127) / 128;
    const int64_t my = (int64_t)blockIdx.x < n_tiles ? (n_tiles - blockIdx.x + gridDim.x - 1) / gridDim.x : 0;
    if (my == 0) return;                         // uniform per CTA: before any setup
    if (tid == 0) {
        for (int i = 0; i < S; i++) {
            mbar_init(smem_u32(&bars[i]), 1);
            mbar_init(smem_u32(&bars[B_CONV + i]), 128);
            mbar_init(smem_u32(&bars[B_EMPTY + i]), 1);
        }
        for (int q = 0; q < 2; q++) {
            mbar_init(smem_u32(&bars[B_ACC + q]), 1);
            mbar_init(smem_u32(&bars[B_ACCE + q]), 128);
        }
        mbar_init(smem_u32(&bars[B_ACT]), 128);
        mbar_init(smem_u32(&bars[B_DRAIN]), 1);
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(a.tmem_cols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;
    const uint32_t act_hi = smem_u32(sm + a.act_off), act_lo = act_hi + (uint32_t)KBW * kABox;

    // The stage sequence every role walks: rounds r = 0 .. my; round r cuts
    // tile r's layer-0 k-blocks into H + 1 chunks and puts tile r - 1's
    // hidden layers 1 .. H between them, so that chain (each layer waits for
    // the epilogue of the one before) overlaps tile r's streaming.
    auto chunk_lo = [&](int c) { return (c * a.nkb0) / (H + 1); };

    if (warp == 0) {
        // ---------------- TMA producer ----------------
        if (lane == 0) {
            asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&amap)) : "memory");
            int slot = 0;
            uint32_t phase = 0, issued_mask = 0, issued_par = 0;
            bool ok = true;
            auto next = [&]() -> bool {
                if (!mbar_wait(smem_u32(&bars[B_EMPTY + slot]), phase ^ 1u, abort_flag, status, wlim)) return false;
                return true;
            };
            auto advance = [&]() {
                issued_mask |= 1u << slot;
                issued_par = (issued_par & ~(1u << slot)) | (phase << slot);
                if (++slot == S) { slot = 0; phase ^= 1u; }
            };
            for (int64_t r = 0; r <= my && ok; r++) {
                const int64_t tile = blockIdx.x + r * gridDim.x;
                for (int c = 0; c <= H && ok; c++) {
                    if (r < my)
                        for (int kb = chunk_lo(c); kb < chunk_lo(c + 1); kb++) {   // layer 0: input rows and W_0
                            if (!(ok = next())) break;
                            const uint32_t fb = smem_u32(&bars[slot]);
                            const uint32_t st = smem_u32(sm + (uint32_t)slot * a.stage_bytes);
                            const uint32_t bh = st + 2u * kABox;
                            mbar_expect_tx(fb, kABox + 2u * (uint32_t)W * 128u);
                            tma_load_2d(st, &amap, kb * 32, (int)(tile * 128), fb);
                            tma_load_2d(bh, &wm.w[0], kb * 32, 0, fb);
                            tma_load_2d(bh + (uint32_t)W * 128u, &wm.w[0], kb * 32, W, fb);
                            advance();
                        }
                    if (c < H && r >= 1 && ok) {
                        const int l = c + 1, rows = l == H ? 16 : W;             // tile r - 1's layer l: its weight
                        for (int kb = 0; kb < KBW; kb++) {
                            if (!(ok = next())) break;
                            const uint32_t fb = smem_u32(&bars[slot]);
                            const uint32_t bh = smem_u32(sm + (uint32_t)slot * a.stage_bytes) + 2u * kABox;
                            mbar_expect_tx(fb, 2u * (uint32_t)rows * 128u);
                            tma_load_2d(bh, &wm.w[l], kb * 32, 0, fb);
                            tma_load_2d(bh + (uint32_t)W * 128u, &wm.w[l], kb * 32, rows, fb);
                            advance();
                        }
                    }
                }
            }
            // every issued copy must have landed before the CTA exits
            for (int i = 0; i < S; i++)
                if (issued_mask >> i & 1u) {
                    volatile int dummy = 0;
                    mbar_wait(smem_u32(&bars[i]), (issued_par >> i) & 1u, &dummy, status);
                }
        }
    } else if (warp == 1) {
        // ---------------- MMA issuer ----------------
        if (lane == 0) {
            const uint32_t id_w = idesc_tf32(W), id_o = idesc_tf32(16);
            int slot = 0;
            uint32_t phase = 0, act_par = 0;
            uint32_t ae_par[2] = {0u, 0u};
            bool ok = true;
            auto take = [&]() -> bool {
                if (!mbar_wait(smem_u32(&bars[B_CONV + slot]), phase, abort_flag, status, wlim)) return false;
                tc_fence_after();
                return true;
            };
            auto release = [&]() {
                mma_commit(smem_u32(&bars[B_EMPTY + slot]));   // frees the stage when these MMAs finish
                if (++slot == S) { slot = 0; phase ^= 1u; }
            };
            for (int64_t r = 0; r <= my && ok; r++) {
                const int qr = (int)(r & 1), qp = (int)((r + 1) & 1);
                const uint32_t acc_r = tmem + (uint32_t)qr * a.acc_stride, acc_p = tmem + (uint32_t)qp * a.acc_stride;
                if (r < my && r >= 2) {   // the epilogue must have read tile r - 2's last layer
                    if (!mbar_wait(smem_u32(&bars[B_ACCE + qr]), ae_par[qr], abort_flag, status, wlim)) { ok = false; break; }
                    ae_par[qr] ^= 1u;
                    tc_fence_after();
                }
                for (int c = 0; c <= H && ok; c++) {
                    if (r < my)
                        for (int kb = chunk_lo(c); kb < chunk_lo(c + 1); kb++) {
                            if (!(ok = take())) break;
                            const uint32_t st = smem_u32(sm + (uint32_t)slot * a.stage_bytes);
                            const uint32_t bh = st + 2u * kABox, bl = bh + (uint32_t)W * 128u;
#pragma unroll
                            for (int ks = 0; ks < 4; ks++)
                                mma_x3(acc_r, st, st + kABox, bh, bl, 32u * ks, id_w, (kb > 0 || ks > 0) ? 1u : 0u);
                            release();
                            if (kb == a.nkb0 - 1) mma_commit(smem_u32(&bars[B_ACC + qr]));   // tile r's layer 0
                        }
                    if (c < H && r >= 1 && ok) {
                        // tile r - 1's layer c + 1 reads the activation tile of its layer c
                        if (!mbar_wait(smem_u32(&bars[B_ACT]), act_par, abort_flag, status, wlim)) { ok = false; break; }
                        act_par ^= 1u;
                        tc_fence_after();
                        const uint32_t id = c + 1 == H ? id_o : id_w;
                        for (int kb = 0; kb < KBW; kb++) {
                            if (!(ok = take())) break;
                            const uint32_t bh = smem_u32(sm + (uint32_t)slot * a.stage_bytes) + 2u * kABox;
                            const uint32_t bl = bh + (uint32_t)W * 128u;
                            const uint32_t ah = act_hi + (uint32_t)kb * kABox, al = act_lo + (uint32_t)kb * kABox;
#pragma unroll
                            for (int ks = 0; ks < 4; ks++)
                                mma_x3(acc_p, ah, al, bh, bl, 32u * ks, id, (kb > 0 || ks > 0) ? 1u : 0u);
                            release();
                        }
                        if (ok) mma_commit(smem_u32(&bars[B_ACC + qp]));
                    }
                }
            }
            // all MMAs of this CTA complete before TMEM is released
            mma_commit(smem_u32(&bars[B_DRAIN]));
            volatile int dummy = 0;
            mbar_wait(smem_u32(&bars[B_DRAIN]), 0, &dummy, status);
        }
    } else if (warp >= 6) {
        // ---------------- splitter: layer-0 A boxes -> hi in place + lo copy ----------------
        const int ct = tid - 192;
        int slot = 0;
        uint32_t phase = 0;
        bool ok = true;
        for (int64_t r = 0; r <= my && ok; r++)
            for (int c = 0; c <= H && ok; c++) {
                const int n0 = r < my ? chunk_lo(c + 1) - chunk_lo(c) : 0;   // layer-0 stages to split
                const int n1 = (c < H && r >= 1) ? KBW : 0;                    // weight-only stages
                for (int u = 0; u < n0 + n1; u++) {
                    if (!mbar_wait(smem_u32(&bars[slot]), phase, abort_flag, status, wlim)) { ok = false; break; }
                    if (u < n0) {
                        float4* A = reinterpret_cast<float4*>(sm + (uint32_t)slot * a.stage_bytes);
                        float4* Al = reinterpret_cast<float4*>(sm + (uint32_t)slot * a.stage_bytes + kABox);
#pragma unroll
                        for (int i = 0; i < 8; i++) {
                            const int idx = ct + 128 * i;
                            float4 hv, lv;
                            split4(A[idx], hv, lv);
                            A[idx] = hv;
                            Al[idx] = lv;
                        }
                        fence_async_smem();
                    }
                    mbar_arrive(smem_u32(&bars[B_CONV + slot]));
                    if (++slot == S) { slot = 0; phase ^= 1u; }
                }
            }
    } else {
        // ---------------- epilogue (warps 2..5) ----------------
        const int qw = warp & 3;                  // TMEM lane quarter this warp may access
        const int r = qw * 32 + lane;             // this thread's row of the tile
        uint8_t* stg = sm + a.stg_off + (uint32_t)(warp - 2) * 4096u;
        uint8_t* ahp = sm + a.act_off;
        uint8_t* alp = ahp + (size_t)KBW * kABox;
        uint32_t af_par[2] = {0u, 0u};
        X3Args so{};
        so.N = W;
        bool ok = true;
        for (int64_t j = 0; j < my && ok; j++) {
            const int q = (int)(j & 1);
            const int64_t tile = blockIdx.x + j * gridDim.x;
            const int64_t row0 = tile * 128 + qw * 32;
            const uint32_t tb = tmem + ((uint32_t)(qw * 32) << 16) + (uint32_t)q * a.acc_stride;
            for (int l = 0; l <= H; l++) {
                int got = 0;
                if (lane == 0) got = mbar_wait(smem_u32(&bars[B_ACC + q]), af_par[q], abort_flag, status, wlim) ? 1 : 0;
                got = __shfl_sync(0xffffffffu, got, 0);
                if (!got) { ok = false; break; }
                af_par[q] ^= 1u;
                tc_fence_after();
                if (l < H) {
                    so.C = a.acts + (int64_t)l * a.n_max * W;
                    so.ldc = W;
#pragma unroll
                    for (int c0 = 0; c0 < W; c0 += 32) {
                        float v[32];
                        tmem_ld32(tb + (uint32_t)c0, v);
#pragma unroll
                        for (int i = 0; i < 32; i++) v[i] = fmaxf(v[i], 0.f);
                        // the next layer's A operand: k-block c0 / 32, split into hi and lo
                        const uint32_t kb = (uint32_t)c0 / 32u;
#pragma unroll
                        for (int ch = 0; ch < 8; ch++) {
                            float4 hv, lv;
                            split4(make_float4(v[4 * ch], v[4 * ch + 1], v[4 * ch + 2], v[4 * ch + 3]), hv, lv);
                            const uint32_t off = kb * kABox + (uint32_t)r * 128u + (uint32_t)((ch ^ (r & 7)) << 4);
                            *reinterpret_cast<float4*>(ahp + off) = hv;
                            *reinterpret_cast<float4*>(alp + off) = lv;
                        }
                        if (a.acts) x3_store<kX3Relu, 32>(so, stg, v, nullptr, lane, row0, n, c0);
                    }
                    fence_async_smem();
                    tc_fence_before();
                    mbar_arrive(smem_u32(&bars[B_ACT]));
                } else {
                    float v[16];
                    tmem_ld16(tb, v);
                    so.C = a.out;
                    so.ldc = NIF_OUT;
                    so.N = 16;
                    x3_store<kX3Store, 16>(so, stg, v, nullptr, lane, row0, n, 0);
                    so.N = W;
                    tc_fence_before();
                    mbar_arrive(smem_u32(&bars[B_ACCE + q]));
                }
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(a.tmem_cols) : "memory");
    }
}

// ---------------------------------------------------------------------------
// Weight gradient of one layer on tensor cores: D = dW_l^T [in_l x out_l] =
// X_l^T dY_l, reduction over the rows. CTA (x, y) owns columns
// [128 x, 128 x + 128) of X_l and the 32-row blocks y, y + gridDim.y, ...
// Warps: 0 TMA, 1 MMA, 2-9 transpose + split (the split is latency-bound
// on dependent shared-memory round trips, hence 8 warps), 2-5 the epilogue.
// ---------------------------------------------------------------------------
constexpr int kDwX3Threads = 320;
constexpr int kDwConv = 256;                   // converter threads

struct DwX3Args {
    float* grad;                      // [out_l][in_l] block of the gradient buffer
    float* part;                      // deterministic mode: [gridDim.y][out_l][in_l] sums of each row range
                                      // (stored, then added in range order); nullptr: added in L2
    int in_l, out_l, MI;              // MI: columns of X_l in one TMA box (<= 128)
    int64_t n_max;
    int raw_stages, op_stages;
    uint32_t raw_bytes, xs_bytes;     // raw stage pitch; X box bytes (MI x 32 FP32), then the dY box (out_l x 32)
    uint32_t raw_tx;                  // bytes the two boxes of a raw stage deliver
    uint32_t op_bytes, op_off;        // operand stage: A hi, A lo (16 KB each), B hi, B lo (out_l x 128 B each)
    uint32_t bar_off, tmem_cols;
};

// One 32-row block: A row i = X_l[r][i0 + i] and B row o = dY_l[r][o] over the
// block's rows r, both split into hi and lo in the K-major swizzled layout;
// rows past the live count (`valid`, checked unless FULL) are zero. Thread ct
// of kDwConv: X column ct % 128, rows 16 (ct / 128) .. +16; dY column ct % OUT,
// row group ct / OUT of G.
template <int OUT, bool FULL>
__device__ __forceinline__ void dw_convert(const float* xs, const float* ds, uint8_t* ah, uint8_t* bh, int MI, int ct,
                                           int valid) {
    uint8_t* al = ah + kABox;
    uint8_t* bl = bh + OUT * 128;
    const int xi = ct & 127, xh = ct >> 7;
    if (xi < MI) {
#pragma unroll
        for (int cc = 0; cc < 4; cc++) {
            const int c = xh * 4 + cc;
            float4 x;
            x.x = (FULL || 4 * c + 0 < valid) ? xs[(4 * c + 0) * MI + xi] : 0.f;
            x.y = (FULL || 4 * c + 1 < valid) ? xs[(4 * c + 1) * MI + xi] : 0.f;
            x.z = (FULL || 4 * c + 2 < valid) ? xs[(4 * c + 2) * MI + xi] : 0.f;
            x.w = (FULL || 4 * c + 3 < valid) ? xs[(4 * c + 3) * MI + xi] : 0.f;
            float4 h, l;
            split4(x, h, l);
            const uint32_t off = (uint32_t)xi * 128u + (uint32_t)((c ^ (xi & 7)) << 4);
            *reinterpret_cast<float4*>(ah + off) = h;
            *reinterpret_cast<float4*>(al + off) = l;
        }
    }
    constexpr int G = (kDwConv / OUT) < 8 ? (kDwConv / OUT) : 8;
    constexpr int C = 32 / G / 4;             // 4-row chunks per thread
    const int o = ct % OUT, g = ct / OUT;
    if (g < G) {
#pragma unroll
        for (int cc = 0; cc < C; cc++) {
            const int c = g * C + cc;
            float4 y;
            y.x = (FULL || 4 * c + 0 < valid) ? ds[(4 * c + 0) * OUT + o] : 0.f;
            y.y = (FULL || 4 * c + 1 < valid) ? ds[(4 * c + 1) * OUT + o] : 0.f;
            y.z = (FULL || 4 * c + 2 < valid) ? ds[(4 * c + 2) * OUT + o] : 0.f;
            y.w = (FULL || 4 * c + 3 < valid) ? ds[(4 * c + 3) * OUT + o] : 0.f;
            float4 h, l;
            split4(y, h, l);
            const uint32_t off = (uint32_t)o * 128u + (uint32_t)((c ^ (o & 7)) << 4);
            *reinterpret_cast<float4*>(bh + off) = h;
            *reinterpret_cast<float4*>(bl + off) = l;
        }
    }
}

template <int OUT>
__global__ void __launch_bounds__(kDwX3Threads, 1)
    k_dw_x3(const __grid_constant__ CUtensorMap xmap, const __grid_constant__ CUtensorMap dmap, DwX3Args a,
            const uint32_t* __restrict__ n_dev, int* __restrict__ status) {
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    const uint64_t wlim = wait_limit(status);   // bound of the work loop's waits
    uint8_t* sm = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int RS = a.raw_stages, OS = a.op_stages;
    uint64_t* bars = reinterpret_cast<uint64_t*>(sm + a.bar_off);
    // [0,RS) raw loaded, [RS,2RS) raw free, then [0,OS) operands ready, [OS,2OS) operands free, then acc full
    const int B_RE = RS, B_OF = 2 * RS, B_OE = 2 * RS + OS, B_ACC = 2 * RS + 2 * OS;
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + B_ACC + 1);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(bars + B_ACC + 2);
    const int64_t n = n_dev ? ((int64_t)*n_dev < a.n_max ? (int64_t)*n_dev : a.n_max) : a.n_max;
    const int64_t nkb = (n + 31) / 32;
    const int64_t my = (int64_t)blockIdx.y < nkb ? (nkb - blockIdx.y + gridDim.y - 1) / gridDim.y : 0;
    if (my == 0) return;                          // nothing to add: leave before any setup
    const int i0 = blockIdx.x * 128;

    if (tid == 0) {
        for (int i = 0; i < RS; i++) {
            mbar_init(smem_u32(&bars[i]), 1);
            mbar_init(smem_u32(&bars[B_RE + i]), kDwConv);
        }
        for (int i = 0; i < OS; i++) {
            mbar_init(smem_u32(&bars[B_OF + i]), kDwConv);
            mbar_init(smem_u32(&bars[B_OE + i]), 1);
        }
        mbar_init(smem_u32(&bars[B_ACC]), 1);
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(a.tmem_cols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    // rows [MI, 128) of the A operands stay zero (X_l narrower than one tile)
    if (a.MI < 128 && warp >= 2) {
        const int ct = tid - 64;
        for (int s = 0; s < OS; s++)
            for (int r = a.MI + ct / 8; r < 128; r += kDwConv / 8) {
                uint8_t* base = sm + a.op_off + (uint32_t)s * a.op_bytes + (uint32_t)r * 128u + (uint32_t)(ct % 8) * 16u;
                *reinterpret_cast<float4*>(base) = make_float4(0.f, 0.f, 0.f, 0.f);
                *reinterpret_cast<float4*>(base + kABox) = make_float4(0.f, 0.f, 0.f, 0.f);
            }
        fence_async_smem();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    if (warp == 0) {
        if (lane == 0 && my > 0) {
            int slot = 0;
            uint32_t phase = 0, issued_mask = 0, issued_par = 0;
            for (int64_t j = 0; j < my; j++) {
                const int64_t kb = blockIdx.y + j * gridDim.y;
                if (!mbar_wait(smem_u32(&bars[B_RE + slot]), phase ^ 1u, abort_flag, status, wlim)) break;
                const uint32_t fb = smem_u32(&bars[slot]);
                const uint32_t st = smem_u32(sm + (uint32_t)slot * a.raw_bytes);
                mbar_expect_tx(fb, a.raw_tx);
                tma_load_2d(st, &xmap, i0, (int)(kb * 32), fb);
                tma_load_2d(st + a.xs_bytes, &dmap, 0, (int)(kb * 32), fb);
                issued_mask |= 1u << slot;
                issued_par = (issued_par & ~(1u << slot)) | (phase << slot);
                if (++slot == RS) { slot = 0; phase ^= 1u; }
            }
            for (int i = 0; i < RS; i++)
                if (issued_mask >> i & 1u) {
                    volatile int dummy = 0;
                    mbar_wait(smem_u32(&bars[i]), (issued_par >> i) & 1u, &dummy, status);
                }
        }
    } else if (warp == 1) {
        if (lane == 0 && my > 0) {
            const uint32_t idesc = idesc_tf32(OUT);
            int slot = 0;
            uint32_t phase = 0;
            for (int64_t j = 0; j < my; j++) {
                if (!mbar_wait(smem_u32(&bars[B_OF + slot]), phase, abort_flag, status, wlim)) break;
                tc_fence_after();
                const uint32_t ah = smem_u32(sm + a.op_off + (uint32_t)slot * a.op_bytes);
                const uint32_t al = ah + kABox, bh = ah + 2u * kABox, bl = bh + (uint32_t)OUT * 128u;
#pragma unroll
                for (int ks = 0; ks < 4; ks++) mma_x3(tmem, ah, al, bh, bl, 32u * ks, idesc, (j > 0 || ks > 0) ? 1u : 0u);
                mma_commit(smem_u32(&bars[B_OE + slot]));
                if (++slot == OS) { slot = 0; phase ^= 1u; }
            }
            mma_commit(smem_u32(&bars[B_ACC]));
            volatile int dummy = 0;
            mbar_wait(smem_u32(&bars[B_ACC]), 0, &dummy, status);
        }
    } else {
        // ---------------- transpose + split (warps 2..9) ----------------
        const int ct = tid - 64;
        int rs = 0, os = 0;
        uint32_t rph = 0, oph = 0;
        for (int64_t j = 0; j < my; j++) {
            const int64_t kb = blockIdx.y + j * gridDim.y;
            if (!mbar_wait(smem_u32(&bars[rs]), rph, abort_flag, status, wlim)) break;
            if (!mbar_wait(smem_u32(&bars[B_OE + os]), oph ^ 1u, abort_flag, status, wlim)) break;
            const float* xs = reinterpret_cast<const float*>(sm + (uint32_t)rs * a.raw_bytes);
            const float* ds = reinterpret_cast<const float*>(sm + (uint32_t)rs * a.raw_bytes + a.xs_bytes);
            uint8_t* ah = sm + a.op_off + (uint32_t)os * a.op_bytes;
            uint8_t* bh = ah + 2u * kABox;
            const int64_t live = n - kb * 32;                 // rows of this block below the live count
            if (live >= 32) dw_convert<OUT, true>(xs, ds, ah, bh, a.MI, ct, 32);
            else dw_convert<OUT, false>(xs, ds, ah, bh, a.MI, ct, (int)live);
            fence_async_smem();
            mbar_arrive(smem_u32(&bars[B_RE + rs]));
            mbar_arrive(smem_u32(&bars[B_OF + os]));
            if (++rs == RS) { rs = 0; rph ^= 1u; }
            if (++os == OS) { os = 0; oph ^= 1u; }
        }
        // epilogue (warps 2..5): TMEM lane i holds D[i][0..OUT) = dW_l[0..OUT)[i0 + i]
        if (my > 0 && warp < 6) {
            int got = 0;
            if (lane == 0) got = mbar_wait(smem_u32(&bars[B_ACC]), 0, abort_flag, status, wlim) ? 1 : 0;
            got = __shfl_sync(0xffffffffu, got, 0);
            if (got && !*abort_flag) {
                tc_fence_after();
                const int qw = warp & 3;
                const int i = i0 + qw * 32 + lane;
                const uint32_t tb = tmem + ((uint32_t)(qw * 32) << 16);
#pragma unroll
                for (int c0 = 0; c0 < OUT; c0 += 16) {
                    float v[16];
                    tmem_ld16(tb + (uint32_t)c0, v);
                    if (i < a.in_l) {
                        if (a.part) {
                            float* p = a.part + ((int64_t)blockIdx.y * a.out_l + c0) * a.in_l + i;
#pragma unroll
                            for (int k = 0; k < 16; k++) p[(int64_t)k * a.in_l] = v[k];
                        } else {
#pragma unroll
                            for (int k = 0; k < 16; k++) atomicAdd(a.grad + (int64_t)(c0 + k) * a.in_l + i, v[k]);
                        }
                    }
                }
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(a.tmem_cols) : "memory");
    }
}

// ---------------------------------------------------------------------------
// hi / lo copies of every layer's weights: forward block [2][out_l][in_l]
// (B of X W_l^T) and transposed block [2][npad_l][out_l] (B of dY W_l; rows
// in_l .. npad_l stay zero)
// ---------------------------------------------------------------------------
struct X3SplitArgs {
    int n;
    int64_t start[NIF_MAX_LAYERS + 1];   // running element count
    int in[NIF_MAX_LAYERS], out[NIF_MAX_LAYERS], npad[NIF_MAX_LAYERS];
    int64_t src[NIF_MAX_LAYERS], fwd[NIF_MAX_LAYERS], bwd[NIF_MAX_LAYERS];
};

__global__ void k_split_weights(const float* __restrict__ params, X3SplitArgs a, float* __restrict__ dst) {
    const int64_t total = a.start[a.n];
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        int l = 0;
        while (e >= a.start[l + 1]) l++;
        const int64_t k = e - a.start[l];
        const int o = (int)(k / a.in[l]), i = (int)(k % a.in[l]);
        float hi, lo;
        split_tf32(params[a.src[l] + k], hi, lo);
        const int64_t nf = (int64_t)a.out[l] * a.in[l], nb = (int64_t)a.npad[l] * a.out[l];
        dst[a.fwd[l] + k] = hi;
        dst[a.fwd[l] + nf + k] = lo;
        dst[a.bwd[l] + (int64_t)i * a.out[l] + o] = hi;
        dst[a.bwd[l] + nb + (int64_t)i * a.out[l] + o] = lo;
    }
}

// N columns in chunks of at most cap (<= 256, one MMA's N): n_chunks and the chunk width NB (a multiple of 16)
void x3_chunks(int N, int* n_chunks, int* NB, int cap = 256) {
    *n_chunks = (N + cap - 1) / cap;
    int w = (N + *n_chunks - 1) / *n_chunks;
    *NB = (w + 15) / 16 * 16;
}

uint32_t pow2_cols(uint32_t c) {
    uint32_t p = 32;
    while (p < c) p <<= 1;
    return p;
}

nif_status map_f32(nif_handle* h, CUtensorMap* map, const void* base, uint64_t inner, uint64_t outer,
                   uint64_t row_elems, uint32_t box_inner, uint32_t box_outer, bool swizzle, const char* what) {
    if ((reinterpret_cast<uintptr_t>(base) & 15) != 0 || (row_elems * 4) % 16 != 0)
        return nif_fail(h, NIF_ERR_ARG, std::string("FP32 MLP: 16-byte aligned rows needed for ") + what);
    cuuint64_t gdim[2] = {(cuuint64_t)inner, (cuuint64_t)outer};
    cuuint64_t gstride[1] = {(cuuint64_t)row_elems * 4};
    cuuint32_t box[2] = {box_inner, box_outer};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = g_encode_tiled(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<void*>(base), gdim, gstride, box,
                                estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                                swizzle ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_NONE,
                                CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return nif_fail(h, NIF_ERR_ARG, std::string("cuTensorMapEncodeTiled failed for ") + what);
    return NIF_OK;
}

// C[r][0..N) = epi(sum_k A[r][k] B[j][k]) for rows r < min(*n_dev, n_max);
// B is the stacked [hi; lo] copy with `npad` rows per copy.
template <int EPI>
nif_status gemm_x3(nif_handle* h, const float* A, int64_t lda, int K, int64_t n_max, const uint32_t* n_dev,
                   const float* B, int N, int npad, float* C, int64_t ldc, const float* mask, int64_t ldm,
                   cudaStream_t s) {
    if (n_max <= 0) return NIF_OK;
    X3Args a{};
    // mask jobs keep two 128 x NB mask tiles in shared memory: NB <= 64
    x3_chunks(N, &a.n_chunks, &a.NB, EPI == kX3Mask ? 64 : 256);
    if (a.n_chunks * a.NB > npad) return nif_fail(h, NIF_ERR_STATE, "FP32 MLP: weight copy narrower than its chunks");
    if (N % 4 != 0 || ldc % 4 != 0 || (reinterpret_cast<uintptr_t>(C) & 15) != 0 ||
        (EPI == kX3Mask && (ldm % 4 != 0 || (reinterpret_cast<uintptr_t>(mask) & 15) != 0)))
        return nif_fail(h, NIF_ERR_ARG, "FP32 MLP: outputs need 16-byte aligned rows");
    CUtensorMap am, bm, mm;
    nif_status st;
    if ((st = map_f32(h, &am, A, (uint64_t)K, (uint64_t)n_max, (uint64_t)lda, 32, 128, true, "the input rows")) != NIF_OK)
        return st;
    if ((st = map_f32(h, &bm, B, (uint64_t)K, 2ull * npad, (uint64_t)K, 32, (uint32_t)a.NB, true, "the weights")) !=
        NIF_OK)
        return st;
    a.mbox = a.NB < 32 ? a.NB : 32;
    if (EPI == kX3Mask) {
        if ((st = map_f32(h, &mm, mask, (uint64_t)N, (uint64_t)n_max, (uint64_t)ldm, (uint32_t)a.mbox, 128, false,
                          "the activations")) != NIF_OK)
            return st;
        a.msk_bytes = 128u * (uint32_t)a.NB * 4u;
    } else {
        mm = am;
        a.msk_bytes = 0;
    }
    a.C = C; a.ldc = ldc; a.mask = mask; a.ldm = ldm;
    a.N = N; a.nkb = (K + 31) / 32; a.n_max = n_max; a.b_lo_row = npad;
    a.b_bytes = (uint32_t)a.NB * 128u;
    a.stage_bytes = 2u * kABox + 2u * a.b_bytes;
    const uint32_t stg = 4u * 4096u, bars = 8u * 64u;
    a.stages = (int)std::min<uint32_t>(4u, (kX3Budget - stg - 2u * a.msk_bytes - bars - 1024u) / a.stage_bytes);
    if (a.stages < 2) return nif_fail(h, NIF_ERR_STATE, "FP32 MLP: pipeline does not fit in shared memory");
    a.stg_off = (uint32_t)a.stages * a.stage_bytes;
    a.msk_off = a.stg_off + stg;
    a.bar_off = a.msk_off + 2u * a.msk_bytes;
    a.acc_stride = pow2_cols((uint32_t)a.NB);
    a.tmem_cols = 2u * a.acc_stride;
    const uint32_t total = a.bar_off + bars + 1024u;
    NIF_CK(h, cudaFuncSetAttribute(k_gemm_x3<EPI>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)total));
    const int64_t jobs = (n_max + 127) / 128 * a.n_chunks;
    const int grid = (int)std::min<int64_t>(jobs, h->num_sms);
    k_gemm_x3<EPI><<<grid, kX3Threads, total, s>>>(am, bm, mm, a, n_dev, h->d_status);
    NIF_CK_LAUNCH(h);
    return NIF_OK;
}

// grad[o][i] += sum_r X[r][i] dY[r][o] over rows r < min(*n_dev, n_max)
nif_status dw_x3(nif_handle* h, const float* X, int64_t ldx, int in_l, const float* dY, int64_t ldy, int out_l,
                 int64_t n_max, const uint32_t* n_dev, float* grad, cudaStream_t s) {
    if (n_max <= 0) return NIF_OK;
    if (out_l < 16 || out_l > 128 || 128 % out_l != 0)
        return nif_fail(h, NIF_ERR_ARG, "FP32 weight gradient: layer width must divide 128");
    DwX3Args a{};
    a.grad = grad; a.in_l = in_l; a.out_l = out_l; a.n_max = n_max;
    a.MI = std::min(128, in_l);
    CUtensorMap xm, dm;
    nif_status st;
    if ((st = map_f32(h, &xm, X, (uint64_t)in_l, (uint64_t)n_max, (uint64_t)ldx, (uint32_t)a.MI, 32, false,
                      "the layer inputs")) != NIF_OK)
        return st;
    if ((st = map_f32(h, &dm, dY, (uint64_t)out_l, (uint64_t)n_max, (uint64_t)ldy, (uint32_t)out_l, 32, false,
                      "the output gradients")) != NIF_OK)
        return st;
    a.xs_bytes = (uint32_t)a.MI * 32u * 4u;
    a.raw_tx = a.xs_bytes + (uint32_t)out_l * 32u * 4u;
    a.raw_bytes = (a.raw_tx + 1023u) & ~1023u;
    a.op_bytes = 2u * kABox + 2u * (uint32_t)out_l * 128u;
    a.op_stages = 2;
    const uint32_t bars = 8u * 32u;
    const uint32_t raw_room = kX3Budget - bars - 1024u - (uint32_t)a.op_stages * a.op_bytes;
    a.raw_stages = (int)std::min<uint32_t>(4u, raw_room / a.raw_bytes);
    if (a.raw_stages < 2) return nif_fail(h, NIF_ERR_STATE, "FP32 weight gradient: pipeline does not fit");
    a.op_off = (uint32_t)a.raw_stages * a.raw_bytes;
    a.bar_off = a.op_off + (uint32_t)a.op_stages * a.op_bytes;
    a.tmem_cols = pow2_cols((uint32_t)out_l);
    const uint32_t total = a.bar_off + bars + 1024u;
    const int tiles = (in_l + 127) / 128;
    const int64_t nkb = (n_max + 31) / 32;
    const int gy = (int)std::max<int64_t>(1, std::min<int64_t>(nkb, std::max(1, h->num_sms / tiles)));
    const int64_t cnt = (int64_t)out_l * in_l;
    if (h->det) {
        // each row range's sum kept apart (a range with no live rows leaves zeros)
        if ((st = nif_grow(h, h->b_parts, sizeof(float) * (size_t)gy * cnt)) != NIF_OK) return st;
        a.part = (float*)h->b_parts.p;
        NIF_CK(h, cudaMemsetAsync(a.part, 0, sizeof(float) * (size_t)gy * cnt, s));
    }
    auto launch = [&](auto kern) -> nif_status {
        NIF_CK(h, cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)total));
        kern<<<dim3(tiles, gy), kDwX3Threads, total, s>>>(xm, dm, a, n_dev, h->d_status);
        return NIF_OK;
    };
    switch (out_l) {
        case 16: st = launch(k_dw_x3<16>); break;
        case 32: st = launch(k_dw_x3<32>); break;
        case 64: st = launch(k_dw_x3<64>); break;
        default: st = launch(k_dw_x3<128>); break;
    }
    if (st != NIF_OK) return st;
    NIF_CK_LAUNCH(h);
    if (a.part) return nif_sum_parts_run(h, a.part, gy, cnt, grad, s);
    return NIF_OK;
}

// The whole forward in one launch (W = 32 or 64): acts [H][n_max][W] (null:
// not stored), out [n_max][NIF_OUT]; ctas > 0 caps the persistent CTAs.
template <int W>
nif_status mlp_fwd_x3_fused(nif_handle* h, const float* x, int64_t n_max, const uint32_t* n_dev, float* acts,
                            float* out, cudaStream_t s, int ctas) {
    X3FwdArgs a{};
    a.acts = acts; a.out = out; a.n_max = n_max;
    a.K0 = h->in_dim; a.W = W; a.H = h->H;
    a.nkb0 = (a.K0 + 31) / 32;
    a.nkbw = W / 32;
    if ((reinterpret_cast<uintptr_t>(acts) & 15) || (reinterpret_cast<uintptr_t>(out) & 15))
        return nif_fail(h, NIF_ERR_ARG, "FP32 MLP: outputs need 16-byte aligned rows");
    CUtensorMap am;
    X3FwdMaps wm{};
    nif_status st;
    if ((st = map_f32(h, &am, x, (uint64_t)a.K0, (uint64_t)n_max, (uint64_t)a.K0, 32, 128, true, "the input rows")) !=
        NIF_OK)
        return st;
    for (int l = 0; l <= a.H; l++) {
        const int K = h->lay_in[l], rows = h->lay_out[l];
        if ((st = map_f32(h, &wm.w[l], h->d_w_x3 + h->x3_fwd[l], (uint64_t)K, 2ull * rows, (uint64_t)K, 32,
                          (uint32_t)rows, true, "the weights")) != NIF_OK)
            return st;
    }
    a.stage_bytes = 2u * kABox + 2u * (uint32_t)W * 128u;
    const uint32_t act = 2u * (uint32_t)a.nkbw * kABox, stg = 4u * 4096u, bars = 8u * 64u;
    const uint32_t budget = 227u * 1024u;
    a.stages = (int)std::min<uint32_t>(4u, (budget - act - stg - bars - 1024u) / a.stage_bytes);
    if (a.stages < 2) return nif_fail(h, NIF_ERR_STATE, "FP32 MLP: fused pipeline does not fit in shared memory");
    a.act_off = (uint32_t)a.stages * a.stage_bytes;
    a.stg_off = a.act_off + act;
    a.bar_off = a.stg_off + stg;
    a.acc_stride = pow2_cols((uint32_t)W);
    a.tmem_cols = 2u * a.acc_stride;
    const uint32_t total = a.bar_off + bars + 1024u;
    NIF_CK(h, cudaFuncSetAttribute(k_mlp_x3_fwd<W>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)total));
    const int64_t tiles = (n_max + 127) / 128;
    const int grid = (int)std::min<int64_t>(tiles, ctas > 0 ? std::min(ctas, h->num_sms) : h->num_sms);
    k_mlp_x3_fwd<W><<<grid, kX3Threads, total, s>>>(am, wm, a, n_dev, h->d_status);
    NIF_CK_LAUNCH(h);
    return NIF_OK;
}

}  // namespace

nif_status nif_x3_alloc(nif_handle* h) {
    size_t off = 0;
    for (int l = 0; l < h->n_layers; l++) {
        int nch, nb;
        x3_chunks(h->lay_in[l], &nch, &nb);
        h->x3_npad[l] = nch * nb;
        h->x3_fwd[l] = off;
        off += 2 * (size_t)h->lay_out[l] * h->lay_in[l];
        off = (off + 3) & ~(size_t)3;
        h->x3_bwd[l] = off;
        off += 2 * (size_t)h->x3_npad[l] * h->lay_out[l];
        off = (off + 3) & ~(size_t)3;
    }
    NIF_CK(h, cudaMalloc(&h->d_w_x3, sizeof(float) * off));
    NIF_CK(h, cudaMemset(h->d_w_x3, 0, sizeof(float) * off));
    h->x3_dirty = true;
    return NIF_OK;
}

nif_status nif_refresh_x3(nif_handle* h, cudaStream_t s) {
    if (!h->x3_dirty) return NIF_OK;
    X3SplitArgs a{};
    a.n = h->n_layers;
    a.start[0] = 0;
    for (int l = 0; l < h->n_layers; l++) {
        a.in[l] = h->lay_in[l];
        a.out[l] = h->lay_out[l];
        a.npad[l] = h->x3_npad[l];
        a.src[l] = (int64_t)h->off_layer[l];
        a.fwd[l] = (int64_t)h->x3_fwd[l];
        a.bwd[l] = (int64_t)h->x3_bwd[l];
        a.start[l + 1] = a.start[l] + (int64_t)a.in[l] * a.out[l];
    }
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(h->num_sms * 4, (a.start[a.n] + 255) / 256));
    k_split_weights<<<grid, 256, 0, s>>>(h->d_params, a, h->d_w_x3);
    NIF_CK_LAUNCH(h);
    h->x3_dirty = false;
    return NIF_OK;
}

nif_status nif_mlp_fwd_fp32_run(nif_handle* h, const float* x, const uint32_t* n_dev, int64_t n_max, float* out,
                                float* acts, cudaStream_t s, int ctas, bool query) {
    NifProf prof_(h, "mlp_fwd_fp32", s);
    if (n_max <= 0) return NIF_OK;
    nif_status st = get_encoder(h);
    if (st != NIF_OK) return st;
    if ((st = nif_refresh_x3(h, s)) != NIF_OK) return st;
    // hidden widths 32 and 64 on request: every layer in one launch, hidden activations on chip
    const bool fusable = (query ? h->tune.query_fp32_fused : h->tune.fp32_fused) && h->H >= 1 &&
                         h->H < NIF_MAX_LAYERS && h->in_dim % 4 == 0;
    float* kept = query ? nullptr : acts;        // a query needs no hidden activations
    if (fusable && h->W == 64) return mlp_fwd_x3_fused<64>(h, x, n_max, n_dev, kept, out, s, ctas);
    if (fusable && h->W == 32) return mlp_fwd_x3_fused<32>(h, x, n_max, n_dev, kept, out, s, ctas);
    const float* in = x;
    int64_t in_ld = h->in_dim;
    for (int l = 0; l < h->n_layers; l++) {
        const float* B = h->d_w_x3 + h->x3_fwd[l];
        const int K = h->lay_in[l], N = h->lay_out[l];
        if (l == h->n_layers - 1) {
            st = gemm_x3<kX3Store>(h, in, in_ld, K, n_max, n_dev, B, N, N, out, NIF_OUT, nullptr, 0, s);
        } else {
            float* dst = acts + (int64_t)l * n_max * h->W;
            st = gemm_x3<kX3Relu>(h, in, in_ld, K, n_max, n_dev, B, N, N, dst, h->W, nullptr, 0, s);
            in = dst;
            in_ld = h->W;
        }
        if (st != NIF_OK) return st;
    }
    return NIF_OK;
}

nif_status nif_mlp_bwd_fp32_run(nif_handle* h, const float* x, const uint32_t* n_dev, int64_t n_max,
                                const float* acts, const float* dout, float* dx, cudaStream_t s, bool want_dw,
                                cudaStream_t aux) {
    if (n_max <= 0) return NIF_OK;
    nif_status st = get_encoder(h);
    if (st != NIF_OK) return st;
    if ((st = nif_refresh_x3(h, s)) != NIF_OK) return st;
    // dY_l of every hidden layer is kept for the weight gradients: [H][n_max][W]
    if ((st = nif_grow(h, h->b_dout, sizeof(float) * (size_t)n_max * h->W * h->H)) != NIF_OK) return st;
    float* dys = (float*)h->b_dout.p;
    const int H = h->H;
    auto dy = [&](int l) { return l == H ? dout : dys + (int64_t)l * n_max * h->W; };
    auto dy_ld = [&](int l) { return l == H ? (int64_t)NIF_OUT : (int64_t)h->W; };
    {
        // dY_{l-1} = (dY_l W_l) * [act_{l-1} > 0]
        NifProf prof_(h, "mlp_bwd_fp32", s);
        for (int l = H; l >= 1; l--) {
            const float* Bt = h->d_w_x3 + h->x3_bwd[l];
            const float* act = acts + (int64_t)(l - 1) * n_max * h->W;
            if ((st = gemm_x3<kX3Mask>(h, dy(l), dy_ld(l), h->lay_out[l], n_max, n_dev, Bt, h->W, h->x3_npad[l],
                                       dys + (int64_t)(l - 1) * n_max * h->W, h->W, act, h->W, s)) != NIF_OK)
                return st;
        }
    }
    cudaStream_t ws = s;
    if (want_dw && aux) {
        // every dY_l is final: the weight gradients overlap dX_0 and what follows
        NIF_CK(h, cudaEventRecord(h->ev_fork, s));
        NIF_CK(h, cudaStreamWaitEvent(aux, h->ev_fork, 0));
        ws = aux;
    }
    if (want_dw) {
        // dW_l += dY_l^T X_l
        NifProf prof_(h, "mlp_dw_fp32", ws);
        for (int l = 0; l <= H; l++) {
            const float* X = l == 0 ? x : acts + (int64_t)(l - 1) * n_max * h->W;
            const int64_t ldx = l == 0 ? h->in_dim : h->W;
            if ((st = dw_x3(h, X, ldx, h->lay_in[l], dy(l), dy_ld(l), h->lay_out[l], n_max, n_dev,
                            h->d_grad + h->off_layer[l], ws)) != NIF_OK)
                return st;
        }
    }
    if (ws != s) NIF_CK(h, cudaEventRecord(h->ev_join, ws));
    if (dx) {
        // dX_0 = dY_0 W_0
        NifProf prof_(h, "mlp_dx_fp32", s);
        if ((st = gemm_x3<kX3Store>(h, dy(0), dy_ld(0), h->lay_out[0], n_max, n_dev, h->d_w_x3 + h->x3_bwd[0],
                                    h->in_dim, h->x3_npad[0], dx, h->in_dim, nullptr, 0, s)) != NIF_OK)
            return st;
    }
    return NIF_OK;
}
