// k_mlp_enc.cu -- the query path's hybrid encoding psi = phi o gamma (Eq. 1)
// and MLP (Sec. 2, Fig. 2d) in one persistent kernel: the features of a
// 128-segment tile are computed by producer warps straight into the
// shared-memory ring that the tensor cores read (tcgen05.mma kind::f16, BF16
// or FP16 operands, FP32 accumulation in TMEM), so they never reach global
// memory. Tables are the FP16 copy, as on the two-kernel path
// (nif_encode_segments + the tensor-core MLP).
//
// Column order. The kernel orders a segment's features [term][end point]
// [level][feature] instead of the library's [end point][term][level][feature]
// and loads layer 0's weights with the same column permutation, so layer 0
// computes the same sum in another order. With L = 4, 8 or 16 levels both end
// points of a term then share a 64-column box, so an entry point that repeats
// the previous segment's exit point bit for bit (two thirds of the segments
// of a ray) is evaluated once and written into both rows of the same stage.
//
// One CTA per SM walks 128-row tiles. Warp roles:
//   warp 0      issues every tcgen05.mma from one thread: layer 0 from the
//               ring's stages, layers >= 1 from the activation tile; layer 0
//               of tile j is issued before layers 1..H of tile j - 1 (two
//               TMEM accumulators), so the producers never wait on the chain;
//   warps 1-4   epilogue: tcgen05.ld of the accumulator, ReLU, 16-bit
//               activation tile in shared memory, and the 16 outputs of a row
//               to global memory as FP32;
//   warps 5..   G producer groups of GW warps. Stage k of the CTA's sequence
//               (tile j, box b: k = j nb0 + b) is filled by group k mod G into
//               ring slot k mod S: the group lists the tile's distinct end
//               points, then each thread takes listed points and evaluates the
//               box's gamma terms for them (all L levels of a term in
//               registers), storing 16-bit features in the 128-byte swizzled
//               K-major layout of the MMA operand.
// Every mbarrier wait is bounded (tc_ptx.cuh). A group's decision to stop is
// taken by one of its threads and shared through shared memory between two
// of its named barriers, so that its threads leave the loop together.
#include <algorithm>

#include "enc_grid.cuh"
#include "nif_internal.cuh"
#include "tc_ptx.cuh"

namespace {

constexpr int kRows = 128;                          // MMA M, rows per tile
constexpr uint32_t kStageBytes = kRows * 128;       // one 128 x 64 box of 16-bit features
constexpr uint32_t kGrpBytes = 768;                 // per group: point list, dup flags, warp sums, decision
constexpr int kLB = 2;                              // levels whose corner loads a producer issues together

struct EncLayout {
    uint32_t wo_off, w0_off, wh_off, a_off, x_off, grp_off, bar_off, total;
    int stages;        // ring depth S
    int nb0;           // 64-column boxes of a tile (terms per box: 16 / L)
    int ks0;           // 16-deep k-steps of layer 0 (K0 / 16)
    int nbw, ksw;      // 64-column blocks and k-steps of a W-wide operand
    uint32_t woff[NIF_MAX_LAYERS];   // element offset of each layer in the 16-bit weight copy
};

// u of gamma term t at p (clamped), with the fast sine and cosine: on the
// 16-bit path the features are rounded to 8 or 11 bits, far above the
// intrinsics' error at |x| <= 2^(F-1)
__device__ __forceinline__ float3 term_u_fast(float3 p, int t) {
    if (t == 0) return p;
    const float f = (float)(1 << ((t - 1) >> 1));
    float sx, cx, sy, cy, sz, cz;
    __sincosf(f * p.x, &sx, &cx);
    __sincosf(f * p.y, &sy, &cy);
    __sincosf(f * p.z, &sz, &cz);
    if ((t - 1) & 1) return make_float3((cx + 1.0f) * 0.5f, (cy + 1.0f) * 0.5f, (cz + 1.0f) * 0.5f);
    return make_float3((sx + 1.0f) * 0.5f, (sy + 1.0f) * 0.5f, (sz + 1.0f) * 0.5f);
}

__device__ __forceinline__ void named_bar(int id, int n) {
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(n) : "memory");
}

// Layer 0's [W x K0] row-major weights into the swizzled K-major layout, with
// the kernel's column order: column c = ((t * 2 + e) * L + l) * 2 + f takes
// the library's column ((e * P + t) * L + l) * 2 + f; columns K0 .. 64 nb0
// are zero.
__device__ void load_weight0_perm(uint8_t* dst, const uint16_t* __restrict__ src, int rows, int K0, int nb0, int L,
                                  int P, int tid, int nthr) {
    const int kpad = nb0 * 64;
    for (int i = tid; i < rows * kpad; i += nthr) {
        const int row = i / kpad, c = i - row * kpad;
        uint16_t v = 0;
        if (c < K0) {
            const int f = c & 1, l = (c >> 1) % L, te = (c >> 1) / L;
            const int e = te & 1, t = te >> 1;
            v = src[(size_t)row * K0 + ((e * P + t) * L + l) * 2 + f];
        }
        *reinterpret_cast<uint16_t*>(dst + swz_off(row, c, rows)) = v;
    }
}

template <int W, int L, int GW, int G>
__global__ void __launch_bounds__((5 + G * GW) * 32, 1)
    k_mlp_enc(GridInfo g, const __half* __restrict__ tab, const nif_linseg* __restrict__ lin, EncLayout lay,
              const uint16_t* __restrict__ wts, int K0, int H, int fmt, int64_t n_max,
              const uint32_t* __restrict__ n_dev, float* __restrict__ out, int* __restrict__ status) {
    constexpr int kGT = GW * 32;                    // threads of a producer group
    constexpr int kThr = (5 + G * GW) * 32;
    constexpr uint32_t kAccCols = W < 32 ? 32 : W;
    static_assert(16 % L == 0 && L >= 4, "16 / L gamma terms per 64-column box, whole 16-byte chunks per item");
    const int64_t n = n_dev ? ((int64_t)*n_dev < n_max ? (int64_t)*n_dev : n_max) : n_max;
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    const uint64_t wlim = wait_limit(status);
    uint8_t* sm = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int S = lay.stages;
    uint64_t* bars = reinterpret_cast<uint64_t*>(sm + lay.bar_off);
    // bars: [0,S) full (a group's kGT threads), [S,2S) empty (MMA commit),
    // 2S+{0,1} acc_full, 2S+{2,3} act (128 epilogue threads), 2S+4 drain
    const int B_ACC = 2 * S, B_ACT = 2 * S + 2, B_DRAIN = 2 * S + 4;
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(sm + lay.bar_off + 8 * (2 * S + 6));
    volatile int* abort_flag = reinterpret_cast<volatile int*>(sm + lay.bar_off + 8 * (2 * S + 6) + 8);
    const int64_t n_tiles = (n + kRows - 1) / kRows;
    const int64_t nt = blockIdx.x < n_tiles ? (n_tiles - blockIdx.x + gridDim.x - 1) / gridDim.x : 0;
    // a CTA without tiles leaves before any barrier, tensor memory or weight
    // load: uniform per CTA
    if (nt == 0) return;

    if (tid == 0) {
        for (int i = 0; i < S; i++) {
            mbar_init(smem_u32(&bars[i]), kGT);
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
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(2 * kAccCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    // resident weights: layer 0 [W x K0] (permuted columns), hidden [W x W] x (H-1), output [16 x W]
    load_weight0_perm(sm + lay.w0_off, wts + lay.woff[0], W, K0, lay.nb0, g.L, g.P, tid, kThr);
    for (int l = 1; l < H; l++)
        load_weight(sm + lay.wh_off + (uint32_t)(l - 1) * lay.nbw * W * 128, wts + lay.woff[l], W, W, tid, kThr);
    load_weight(sm + lay.wo_off, wts + lay.woff[H], 16, W, tid, kThr);
    fence_async_smem();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;
    const uint32_t a_bytes = (uint32_t)lay.nbw * kRows * 128;   // one activation tile

    if (warp == 0) {
        // ---------------- MMA issuer ----------------
        if (lane == 0) {
            const uint32_t id_hid = idesc_f16(fmt, W);
            const uint32_t id_out = idesc_f16(fmt, 16);
            uint32_t act_par[2] = {0u, 0u};
            bool ok = true;
            for (int64_t j = 0; j <= nt && ok; j++) {
                if (j < nt) {
                    // layer 0 of tile j
                    const int q = (int)(j & 1);
                    const uint32_t acc = tmem + (uint32_t)q * kAccCols;
                    if (j >= 2) {       // the epilogue has read this accumulator's last layer of tile j - 2
                        if (!mbar_wait(smem_u32(&bars[B_ACT + q]), act_par[q], abort_flag, status, wlim)) { ok = false; break; }
                        act_par[q] ^= 1u;
                        tc_fence_after();
                    }
                    for (int b = 0; b < lay.nb0; b++) {
                        const int64_t k = j * lay.nb0 + b;
                        const int slot = (int)(k % S);
                        const uint32_t ph = (uint32_t)((k / S) & 1);
                        if (!mbar_wait(smem_u32(&bars[slot]), ph, abort_flag, status, wlim)) { ok = false; break; }
                        tc_fence_after();
                        const uint32_t base = smem_u32(sm + lay.x_off + (uint32_t)slot * kStageBytes);
                        const uint32_t wbase = smem_u32(sm + lay.w0_off + (uint32_t)b * W * 128);
                        for (int jj = 0; jj < 4; jj++) {
                            const int ks = b * 4 + jj;
                            if (ks >= lay.ks0) break;
                            mma_f16(acc, sdesc(base + 32 * jj), sdesc(wbase + 32 * jj), id_hid, ks > 0 ? 1u : 0u);
                        }
                        mma_commit(smem_u32(&bars[S + slot]));   // frees the slot when these MMAs finish
                    }
                    if (!ok) break;
                    mma_commit(smem_u32(&bars[B_ACC + q]));
                }
                if (j >= 1) {
                    // layers 1..H of tile j - 1, from the activation tile of its accumulator
                    const int qp = (int)((j - 1) & 1);
                    const uint32_t acc = tmem + (uint32_t)qp * kAccCols;
                    for (int l = 1; l <= H; l++) {
                        if (!mbar_wait(smem_u32(&bars[B_ACT + qp]), act_par[qp], abort_flag, status, wlim)) { ok = false; break; }
                        act_par[qp] ^= 1u;
                        tc_fence_after();
                        const bool last = l == H;
                        const uint32_t wb = last ? smem_u32(sm + lay.wo_off)
                                                 : smem_u32(sm + lay.wh_off + (uint32_t)(l - 1) * lay.nbw * W * 128);
                        const uint32_t ab = smem_u32(sm + lay.a_off + (uint32_t)qp * a_bytes);
                        for (int ks = 0; ks < lay.ksw; ks++) {
                            const uint32_t blk = (uint32_t)(ks >> 2), jj = (uint32_t)(ks & 3);
                            const uint32_t aoff = blk * kRows * 128 + 32 * jj;
                            const uint32_t boff = blk * (uint32_t)(last ? 16 : W) * 128 + 32 * jj;
                            mma_f16(acc, sdesc(ab + aoff), sdesc(wb + boff), last ? id_out : id_hid, ks > 0 ? 1u : 0u);
                        }
                        mma_commit(smem_u32(&bars[B_ACC + qp]));
                    }
                }
            }
            // all MMAs of this CTA complete before TMEM is released
            mma_commit(smem_u32(&bars[B_DRAIN]));
            volatile int dummy = 0;
            mbar_wait(smem_u32(&bars[B_DRAIN]), 0, &dummy, status);
        }
    } else if (warp <= 4) {
        // ---------------- epilogue (warps 1..4), tiles in order ----------------
        const int qw = warp & 3;                  // TMEM lane quarter this warp may access
        const int row = qw * 32 + lane;
        uint32_t acc_par[2] = {0u, 0u};
        bool ok = true;
        for (int64_t j = 0; j < nt && ok; j++) {
            const int q = (int)(j & 1);
            const int64_t grow = ((int64_t)blockIdx.x + j * gridDim.x) * kRows + row;
            for (int l = 0; l <= H; l++) {
                int got = 0;
                if (lane == 0) got = mbar_wait(smem_u32(&bars[B_ACC + q]), acc_par[q], abort_flag, status, wlim) ? 1 : 0;
                got = __shfl_sync(0xffffffffu, got, 0);
                if (!got) { ok = false; break; }
                acc_par[q] ^= 1u;
                tc_fence_after();
                const uint32_t lane_base = tmem + ((uint32_t)(qw * 32) << 16) + (uint32_t)q * kAccCols;
                if (l < H) {
                    uint8_t* A = sm + lay.a_off + (uint32_t)q * a_bytes;
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
                        }
                    }
                    fence_async_smem();
                } else {
                    float v[16];
                    tmem_ld16(lane_base, v);
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
    } else {
        // ---------------- producers: G groups of GW warps ----------------
        const int pw = warp - 5;
        const int grp = pw / GW;
        const int gt = (pw - grp * GW) * 32 + lane;
        uint8_t* gbase = sm + lay.grp_off + (uint32_t)grp * kGrpBytes;
        uint16_t* list = reinterpret_cast<uint16_t*>(gbase);               // <= 256 (row | e << 7 | twice << 8)
        uint8_t* dupf = gbase + 512;                                        // [128] entry repeats the previous exit
        int* wsum = reinterpret_cast<int*>(gbase + 640);                    // [GW] warp totals
        volatile int* gdec = reinterpret_cast<volatile int*>(gbase + 640 + 4 * GW);   // group decision
        const int bar_id = 1 + grp;
        constexpr int kTpb = 16 / L;            // gamma terms per 64-column box
        constexpr int kCpi = L / 4;             // 16-byte chunks of one (point, term) item
        constexpr int R = (kRows + kGT - 1) / kGT;   // tile rows per thread in the listing
        const int64_t n_seq = nt * lay.nb0;
        for (int64_t k = grp; k < n_seq; k += G) {
            const int64_t j = k / lay.nb0;
            const int b = (int)(k - j * lay.nb0);
            const int slot = (int)(k % S);
            const uint32_t ph = (uint32_t)((k / S) & 1);
            const int64_t row0 = ((int64_t)blockIdx.x + j * gridDim.x) * kRows;
            if (gt == 0) *gdec = mbar_wait(smem_u32(&bars[S + slot]), ph ^ 1u, abort_flag, status, wlim) ? 1 : 0;
            named_bar(bar_id, kGT);
            if (!*gdec) break;
            // the tile's distinct end points, in row order: every exit point,
            // and the entry points that do not repeat the previous row's exit
            int cnt = 0;
            bool valid[R], need0[R];
#pragma unroll
            for (int i = 0; i < R; i++) {
                const int r = gt * R + i;
                const int64_t s = row0 + r;
                valid[i] = r < kRows && s < n;
                bool dup = false;
                if (valid[i] && r > 0) {
                    const float* a = reinterpret_cast<const float*>(lin + s);
                    const float* pb = reinterpret_cast<const float*>(lin + s - 1) + 3;
                    dup = a[0] == pb[0] && a[1] == pb[1] && a[2] == pb[2];
                }
                if (r < kRows) dupf[r] = dup ? 1 : 0;
                need0[i] = valid[i] && !dup;
                cnt += (need0[i] ? 1 : 0) + (valid[i] ? 1 : 0);
            }
            int x = cnt;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(0xffffffffu, x, o);
                if (lane >= o) x += y;
            }
            if (lane == 31) wsum[gt >> 5] = x;
            named_bar(bar_id, kGT);
            int pos = x - cnt, m = 0;
#pragma unroll
            for (int w = 0; w < GW; w++) {
                if (w < (gt >> 5)) pos += wsum[w];
                m += wsum[w];
            }
#pragma unroll
            for (int i = 0; i < R; i++) {
                const int r = gt * R + i;
                if (!valid[i]) continue;
                if (need0[i]) list[pos++] = (uint16_t)r;
                const bool twice = r + 1 < kRows && dupf[r + 1];
                list[pos++] = (uint16_t)(r | (1 << 7) | (twice ? 1 << 8 : 0));
            }
            named_bar(bar_id, kGT);
            // the box's terms for every listed point: a thread keeps its points
            // and walks the box's terms
            const int t0 = b * kTpb;
            const int nterm = min(kTpb, g.P - t0);
            uint8_t* stage = sm + lay.x_off + (uint32_t)slot * kStageBytes;
            for (int pi = gt; pi < m; pi += kGT) {
                const uint32_t info = list[pi];
                const int r = (int)(info & 127u), e = (int)((info >> 7) & 1u);
                const bool twice = (info >> 8) & 1u;
                const float* pp = reinterpret_cast<const float*>(lin + row0 + r) + 3 * e;
                const float3 p = clamp01(make_float3(pp[0], pp[1], pp[2]));
                uint8_t* dst = stage + (uint32_t)r * 128u;
                uint8_t* dst2 = dst + 128;
                const int sw = r & 7, sw2 = (r + 1) & 7;
#pragma unroll 1
                for (int tt = 0; tt < nterm; tt++) {
                    const float3 u = term_u_fast(p, t0 + tt);
                    uint32_t res[L];
                    // kLB levels at a time: their 8 kLB corner loads in flight together
#pragma unroll
                    for (int l0 = 0; l0 < L; l0 += kLB) {
                        Cell c[kLB];
                        typename RawRow<__half>::T vr[kLB][8];
#pragma unroll
                        for (int i = 0; i < kLB; i++) {
                            c[i] = cell_of(u, g.res[l0 + i]);
                            level_gather<__half>(g, tab, l0 + i, c[i], vr[i]);
                        }
#pragma unroll
                        for (int i = 0; i < kLB; i++) {
                            // corner weights (x fastest), then both features of a
                            // corner in one packed FP32 FMA
                            const float2 wx = make_float2(1.f - c[i].wx, c[i].wx);
                            const float wy0 = 1.f - c[i].wy, wy1 = c[i].wy, wz0 = 1.f - c[i].wz, wz1 = c[i].wz;
                            const float2 wxy0 = __fmul2_rn(wx, make_float2(wy0, wy0));
                            const float2 wxy1 = __fmul2_rn(wx, make_float2(wy1, wy1));
                            const float2 wq[4] = {__fmul2_rn(wxy0, make_float2(wz0, wz0)),
                                                  __fmul2_rn(wxy1, make_float2(wz0, wz0)),
                                                  __fmul2_rn(wxy0, make_float2(wz1, wz1)),
                                                  __fmul2_rn(wxy1, make_float2(wz1, wz1))};
                            float2 acc = make_float2(0.f, 0.f);
#pragma unroll
                            for (int q = 0; q < 8; q++) {
                                const float w = (q & 1) ? wq[q >> 1].y : wq[q >> 1].x;
                                acc = __ffma2_rn(make_float2(w, w), RawRow<__half>::f2(vr[i][q]), acc);
                            }
                            res[l0 + i] = pack2(acc.x, acc.y, fmt);
                        }
                    }
                    // row r's (term, e) columns; an exit point that the next row
                    // repeats also goes to that row's (term, entry) columns
                    const int c0 = (tt * 2 + e) * kCpi, c2 = tt * 2 * kCpi;
#pragma unroll
                    for (int qc = 0; qc < kCpi; qc++) {
                        const uint4 v4 = make_uint4(res[4 * qc], res[4 * qc + 1], res[4 * qc + 2], res[4 * qc + 3]);
                        *reinterpret_cast<uint4*>(dst + (((c0 + qc) ^ sw) << 4)) = v4;
                        if (twice) *reinterpret_cast<uint4*>(dst2 + (((c2 + qc) ^ sw2) << 4)) = v4;
                    }
                }
            }
            fence_async_smem();
            mbar_arrive(smem_u32(&bars[slot]));
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(2 * kAccCols) : "memory");
    }
}

// shared-memory layout; stages = 0 when the weights leave no room for G + 1 stages
EncLayout make_enc_layout(int W, int K0, int H, int P, int L, int G) {
    EncLayout y{};
    const int tpb = 16 / L;
    y.nb0 = (P + tpb - 1) / tpb;
    y.ks0 = K0 / 16;
    y.nbw = (W + 63) / 64;
    y.ksw = W / 16;
    uint32_t off = 0;
    y.wo_off = off;
    off += (uint32_t)y.nbw * 16 * 128;
    y.w0_off = off;
    off += (uint32_t)y.nb0 * W * 128;
    y.wh_off = off;
    off += (uint32_t)(H - 1) * y.nbw * W * 128;
    off = (off + 1023) & ~1023u;
    y.a_off = off;
    off += 2u * (uint32_t)y.nbw * kRows * 128;      // one activation tile per accumulator
    y.x_off = off;
    const uint32_t fixed = off + (uint32_t)G * kGrpBytes + 8 * (2 * 12 + 6) + 16 + 1024;
    const uint32_t budget = 227 * 1024;
    int S = fixed < budget ? (int)((budget - fixed) / kStageBytes) : 0;
    S = std::min(S, G + 2);
    y.stages = S >= G + 1 ? S : 0;
    off += (uint32_t)std::max(S, 0) * kStageBytes;
    y.grp_off = off;
    off += (uint32_t)G * kGrpBytes;
    y.bar_off = off;
    off += 8 * (2 * std::max(S, 1) + 6) + 16;
    y.total = off + 1024;        // room to align the dynamic buffer to 1024 bytes
    return y;
}

template <int W, int L, int GW, int G>
nif_status launch_enc(nif_handle* h, const nif_linseg* lin, const uint32_t* n_dev, int64_t n_max, float* out,
                      cudaStream_t s) {
    EncLayout lay = make_enc_layout(W, h->in_dim, h->H, h->P, h->L, G);
    if (lay.stages == 0) return nif_fail(h, NIF_ERR_STATE, "fused encoding + MLP: weights leave no room for the ring");
    for (int l = 0; l < h->n_layers; l++) {
        lay.woff[l] = (uint32_t)(h->off_layer[l] - h->off_layer[0]);
        if (lay.woff[l] % 8) return nif_fail(h, NIF_ERR_STATE, "weight copy not 16-byte aligned per layer");
    }
    NIF_CK(h, cudaFuncSetAttribute(k_mlp_enc<W, L, GW, G>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   (int)lay.total));
    const int64_t n_tiles = (n_max + kRows - 1) / kRows;
    const int grid = (int)std::min<int64_t>(n_tiles, h->num_sms);
    const int fmt = h->cfg.precision == NIF_BF16 ? 1 : 0;
    const uint16_t* w = reinterpret_cast<const uint16_t*>(fmt ? (const void*)h->d_w_bf16 : (const void*)h->d_w_f16);
    k_mlp_enc<W, L, GW, G><<<grid, (5 + G * GW) * 32, lay.total, s>>>(
        h->grid, h->d_tables_h, lin, lay, w, h->in_dim, h->H, fmt, n_max, n_dev, out, h->d_status);
    NIF_CK_LAUNCH(h);
    return NIF_OK;
}

// producer groups: 4 groups of 6 warps. A box holds 16 / L terms of the
// tile's ~170 distinct points (2/3 of the entry points repeat an exit), so a
// group of 192 threads walks each term's points in one round
constexpr int kG = 4;
constexpr int kGW = 6;

}  // namespace

// Tables above 4 MiB (FP16 copy) miss L1 at every hashed level, and the 24
// producer warps of a CTA do not hide the L2 latency that the two-kernel
// path's encoder hides with many more warps and rest-space-sorted points
// (measured: 64 instances, 32 MiB tables, 112.8 ms fused against 42.4 ms).
constexpr size_t kFusedTableBytes = (size_t)4 << 20;

bool nif_mlp_enc_fusable(const nif_handle* h) {
    if (!h->tune.query_fused || h->concat || h->Fd != 2) return false;
    if ((size_t)h->T * h->L * h->Fd * sizeof(__half) > kFusedTableBytes) return false;
    if (h->cfg.precision != NIF_BF16 && h->cfg.precision != NIF_FP16) return false;
    if (h->L != 4 && h->L != 8 && h->L != 16) return false;
    if (h->W != 32 && h->W != 64) return false;
    if (h->H < 1 || h->H >= NIF_MAX_LAYERS || h->in_dim != 4 * h->P * h->L) return false;
    return make_enc_layout(h->W, h->in_dim, h->H, h->P, h->L, kG).stages > 0;
}

nif_status nif_mlp_enc_tc_run(nif_handle* h, const nif_linseg* lin, const uint32_t* n_dev, int64_t n_max, float* out,
                              cudaStream_t s) {
    NifProf prof_(h, "encode_mlp_tc", s);
    if (n_max <= 0) return NIF_OK;
    if (!nif_mlp_enc_fusable(h)) return nif_fail(h, NIF_ERR_STATE, "fused encoding + MLP does not apply to this handle");
    nif_status st = nif_refresh_lowp(h, s);
    if (st != NIF_OK) return st;
    switch (h->L * 100 + h->W) {
        case 432: return launch_enc<32, 4, kGW, kG>(h, lin, n_dev, n_max, out, s);
        case 464: return launch_enc<64, 4, kGW, kG>(h, lin, n_dev, n_max, out, s);
        case 832: return launch_enc<32, 8, kGW, kG>(h, lin, n_dev, n_max, out, s);
        case 864: return launch_enc<64, 8, kGW, kG>(h, lin, n_dev, n_max, out, s);
        case 1632: return launch_enc<32, 16, kGW, kG>(h, lin, n_dev, n_max, out, s);
        default: return launch_enc<64, 16, kGW, kG>(h, lin, n_dev, n_max, out, s);
    }
}
