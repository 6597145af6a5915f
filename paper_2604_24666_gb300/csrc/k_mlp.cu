// k_mlp.cu -- FP32 (FFMA) path of the MLP (Sec. 2, Fig. 2d): H hidden ReLU
// layers without bias and a linear output layer, forward and backward.
//
// All products are one tiled SGEMM kernel C = A * B with arbitrary element
// strides (so the same kernel serves X W^T, dY W and dY^T X), 64x64 output
// tiles, 16-deep K slices staged in shared memory, 4x4 outputs per thread,
// and an epilogue chosen per call: store, ReLU, ReLU-derivative mask, or
// split-K atomic accumulation (for weight gradients summed over rows).
#include <algorithm>

#include "nif_internal.cuh"

namespace {

enum Epi { kStore = 0, kRelu = 1, kMask = 2, kAtomic = 3 };

struct GemmArgs {
    const float* A; int64_t sai, sak;     // A(i,k) = A[i*sai + k*sak]
    const float* B; int64_t sbk, sbj;     // B(k,j) = B[k*sbk + j*sbj]
    float* C; int64_t ldc;                // C(i,j) = C[i*ldc + j]
    const float* mask;                    // mask(i,j) = mask[i*ldc + j] (kMask)
    int64_t M; int N; int64_t K;
    const uint32_t* M_dev;                // if set, rows = min(*M_dev, M) (M is rows of C or, for
    int m_is_k;                           //  split-K, rows of the reduction when m_is_k = 1)
    int64_t k_chunk;                      // split-K chunk (kAtomic)
};

constexpr int BM = 64, BN = 64, BK = 16;

template <int EPI>
__global__ void __launch_bounds__(256) k_sgemm(GemmArgs a) {
    __shared__ float sA[BK][BM + 4];
    __shared__ float sB[BK][BN + 4];
    int64_t M = a.M, K = a.K;
    if (a.M_dev) {
        int64_t m = (int64_t)*a.M_dev;
        if (a.m_is_k) K = m < K ? m : K;
        else M = m < M ? m : M;
    }
    int64_t i0 = (int64_t)blockIdx.y * BM;
    int j0 = blockIdx.x * BN;
    if (i0 >= M) return;
    int64_t kb = 0, ke = K;
    if (EPI == kAtomic) {
        kb = (int64_t)blockIdx.z * a.k_chunk;
        ke = kb + a.k_chunk < K ? kb + a.k_chunk : K;
        if (kb >= ke) return;
    }
    int tid = threadIdx.x;
    int tx = tid & 15, ty = tid >> 4;   // 16 x 16 threads, 4x4 outputs each
    float acc[4][4] = {};
    bool a_krow = a.sak == 1;            // A contiguous along k
    bool b_jrow = a.sbj == 1;            // B contiguous along j
    for (int64_t k0 = kb; k0 < ke; k0 += BK) {
#pragma unroll
        for (int e = 0; e < 4; e++) {
            int idx = tid * 4 + e;       // 0..1023
            int ii, kk;
            if (a_krow) { ii = idx / BK; kk = idx % BK; } else { kk = idx / BM; ii = idx % BM; }
            int64_t gi = i0 + ii, gk = k0 + kk;
            sA[kk][ii] = (gi < M && gk < ke) ? a.A[gi * a.sai + gk * a.sak] : 0.f;
            int jj, kk2;
            if (b_jrow) { kk2 = idx / BN; jj = idx % BN; } else { jj = idx / BK; kk2 = idx % BK; }
            int64_t gj = j0 + jj, gk2 = k0 + kk2;
            sB[kk2][jj] = (gj < a.N && gk2 < ke) ? a.B[gk2 * a.sbk + gj * a.sbj] : 0.f;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < BK; kk++) {
            float av[4], bv[4];
#pragma unroll
            for (int r = 0; r < 4; r++) av[r] = sA[kk][ty * 4 + r];
#pragma unroll
            for (int c = 0; c < 4; c++) bv[c] = sB[kk][tx * 4 + c];
#pragma unroll
            for (int r = 0; r < 4; r++)
#pragma unroll
                for (int c = 0; c < 4; c++) acc[r][c] += av[r] * bv[c];
        }
        __syncthreads();
    }
#pragma unroll
    for (int r = 0; r < 4; r++) {
        int64_t gi = i0 + ty * 4 + r;
        if (gi >= M) continue;
#pragma unroll
        for (int c = 0; c < 4; c++) {
            int gj = j0 + tx * 4 + c;
            if (gj >= a.N) continue;
            float v = acc[r][c];
            float* dst = a.C + gi * a.ldc + gj;
            if (EPI == kStore) *dst = v;
            else if (EPI == kRelu) *dst = fmaxf(v, 0.f);
            else if (EPI == kMask) *dst = a.mask[gi * a.ldc + gj] > 0.f ? v : 0.f;
            else atomicAdd(dst, v);
        }
    }
}

// Register-blocked SGEMM for the large products (N a multiple of 64, K a
// multiple of 16 apart from a device-side tail): BMT x 64 output tile, 16-deep
// K slices double-buffered in shared memory (k-major, so each thread reads
// its rows and columns as float4), fed by float4 global loads held in
// registers while the previous slice is multiplied; each of the 256 threads
// owns a (BMT/16) x 4 block of outputs.
template <int EPI, int BMT>
__global__ void __launch_bounds__(256) k_sgemm_big(GemmArgs a) {
    constexpr int BNT = 64, BKT = 16, TM = BMT / 16, LA = BMT / 16;
    __shared__ __align__(16) float sA[2][BKT][BMT];
    __shared__ __align__(16) float sB[2][BKT][BNT];
    int64_t M = a.M, K = a.K;
    if (a.M_dev) {
        int64_t m = (int64_t)*a.M_dev;
        if (a.m_is_k) K = m < K ? m : K;
        else M = m < M ? m : M;
    }
    const int64_t i0 = (int64_t)blockIdx.y * BMT;
    const int j0 = blockIdx.x * BNT;
    if (i0 >= M) return;
    int64_t kb = 0, ke = K;
    if (EPI == kAtomic) {
        kb = (int64_t)blockIdx.z * a.k_chunk;
        ke = kb + a.k_chunk < K ? kb + a.k_chunk : K;
        if (kb >= ke) return;
    }
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    const bool a_krow = a.sak == 1;
    const bool b_jrow = a.sbj == 1;
    // global -> register staging of one K slice
    float ra[LA], rb[4];
    auto load_slice = [&](int64_t k0) {
        const bool full = k0 + BKT <= ke;
        if (a_krow) {
            const int row = tid / (BKT / LA), kk = (tid % (BKT / LA)) * LA;
            const int64_t gi = i0 + row;
            const float* src = a.A + gi * a.sai + (k0 + kk);
#pragma unroll
            for (int q = 0; q < LA; q += 4) {
                float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
                if (gi < M) {
                    if (full) v = *reinterpret_cast<const float4*>(src + q);
                    else {
                        if (k0 + kk + q + 0 < ke) v.x = src[q + 0];
                        if (k0 + kk + q + 1 < ke) v.y = src[q + 1];
                        if (k0 + kk + q + 2 < ke) v.z = src[q + 2];
                        if (k0 + kk + q + 3 < ke) v.w = src[q + 3];
                    }
                }
                ra[q] = v.x; ra[q + 1] = v.y; ra[q + 2] = v.z; ra[q + 3] = v.w;
            }
        } else {
            const int k = tid / 16, ii = (tid % 16) * LA;
            const bool kin = k0 + k < ke;
#pragma unroll
            for (int q = 0; q < LA; q += 4) {
                float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
                const int64_t gi = i0 + ii + q;
                const float* src = a.A + gi + (k0 + k) * a.sak;
                if (kin) {
                    if (gi + 3 < M) v = *reinterpret_cast<const float4*>(src);
                    else {
                        if (gi + 0 < M) v.x = src[0];
                        if (gi + 1 < M) v.y = src[1];
                        if (gi + 2 < M) v.z = src[2];
                    }
                }
                ra[q] = v.x; ra[q + 1] = v.y; ra[q + 2] = v.z; ra[q + 3] = v.w;
            }
        }
        if (b_jrow) {
            const int k = tid / 16, jj = (tid % 16) * 4;
            float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
            if (k0 + k < ke) v = *reinterpret_cast<const float4*>(a.B + (k0 + k) * a.sbk + (j0 + jj));
            rb[0] = v.x; rb[1] = v.y; rb[2] = v.z; rb[3] = v.w;
        } else {
            const int j = tid / 4, kk = (tid % 4) * 4;
            const float* src = a.B + (int64_t)(j0 + j) * a.sbj + (k0 + kk);
            float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
            if (full) v = *reinterpret_cast<const float4*>(src);
            else {
                if (k0 + kk + 0 < ke) v.x = src[0];
                if (k0 + kk + 1 < ke) v.y = src[1];
                if (k0 + kk + 2 < ke) v.z = src[2];
                if (k0 + kk + 3 < ke) v.w = src[3];
            }
            rb[0] = v.x; rb[1] = v.y; rb[2] = v.z; rb[3] = v.w;
        }
    };
    auto store_slice = [&](int buf) {
        if (a_krow) {
            const int row = tid / (BKT / LA), kk = (tid % (BKT / LA)) * LA;
#pragma unroll
            for (int q = 0; q < LA; q++) sA[buf][kk + q][row] = ra[q];
        } else {
            const int k = tid / 16, ii = (tid % 16) * LA;
#pragma unroll
            for (int q = 0; q < LA; q += 4)
                *reinterpret_cast<float4*>(&sA[buf][k][ii + q]) = make_float4(ra[q], ra[q + 1], ra[q + 2], ra[q + 3]);
        }
        if (b_jrow) {
            const int k = tid / 16, jj = (tid % 16) * 4;
            *reinterpret_cast<float4*>(&sB[buf][k][jj]) = make_float4(rb[0], rb[1], rb[2], rb[3]);
        } else {
            const int j = tid / 4, kk = (tid % 4) * 4;
#pragma unroll
            for (int q = 0; q < 4; q++) sB[buf][kk + q][j] = rb[q];
        }
    };
    float acc[TM][4];
#pragma unroll
    for (int r = 0; r < TM; r++)
#pragma unroll
        for (int c = 0; c < 4; c++) acc[r][c] = 0.f;
    load_slice(kb);
    store_slice(0);
    __syncthreads();
    int buf = 0;
    for (int64_t k0 = kb; k0 < ke; k0 += BKT) {
        const bool more = k0 + BKT < ke;
        if (more) load_slice(k0 + BKT);
#pragma unroll
        for (int kk = 0; kk < BKT; kk++) {
            float av[TM];
#pragma unroll
            for (int r = 0; r < TM; r += 4) {
                float4 v = *reinterpret_cast<const float4*>(&sA[buf][kk][ty * TM + r]);
                av[r] = v.x; av[r + 1] = v.y; av[r + 2] = v.z; av[r + 3] = v.w;
            }
            float4 bv = *reinterpret_cast<const float4*>(&sB[buf][kk][tx * 4]);
#pragma unroll
            for (int r = 0; r < TM; r++) {
                acc[r][0] += av[r] * bv.x;
                acc[r][1] += av[r] * bv.y;
                acc[r][2] += av[r] * bv.z;
                acc[r][3] += av[r] * bv.w;
            }
        }
        if (more) {
            store_slice(buf ^ 1);
            __syncthreads();
            buf ^= 1;
        }
    }
#pragma unroll
    for (int r = 0; r < TM; r++) {
        const int64_t gi = i0 + ty * TM + r;
        if (gi >= M) continue;
        const int gj = j0 + tx * 4;
        float* dst = a.C + gi * a.ldc + gj;
        if (EPI == kAtomic) {
#pragma unroll
            for (int c = 0; c < 4; c++) atomicAdd(dst + c, acc[r][c]);
            continue;
        }
        float4 v = make_float4(acc[r][0], acc[r][1], acc[r][2], acc[r][3]);
        if (EPI == kRelu) {
            v.x = fmaxf(v.x, 0.f); v.y = fmaxf(v.y, 0.f); v.z = fmaxf(v.z, 0.f); v.w = fmaxf(v.w, 0.f);
        } else if (EPI == kMask) {
            float4 m = *reinterpret_cast<const float4*>(a.mask + gi * a.ldc + gj);
            v.x = m.x > 0.f ? v.x : 0.f; v.y = m.y > 0.f ? v.y : 0.f;
            v.z = m.z > 0.f ? v.z : 0.f; v.w = m.w > 0.f ? v.w : 0.f;
        }
        *reinterpret_cast<float4*>(dst) = v;
    }
}

// Register-tiled SGEMM, 8 x 8 outputs per thread: BM x 64 block tile
// ((BM/8) x 8 threads), 16-deep K slices double-buffered in shared memory
// (k-major), the next slice held in registers while the current one is
// multiplied. Per k a thread reads two float4 of A and two of B and issues 64
// FMAs, so shared-memory traffic stays well below the FMA rate. Serves
// N % 64 == 0 with A contiguous along k or i and B along j or k.
template <int EPI, int BMR>
__global__ void __launch_bounds__(BMR) k_sgemm_rt(GemmArgs a) {
    constexpr int BNR = 64, BKR = 16, T8 = 8, NT = BMR;          // (BMR/8) x (64/8) threads
    constexpr int A4 = BMR * BKR / 4 / NT, B4 = BKR * BNR / 4 / NT;  // float4 per thread per slice
    __shared__ __align__(16) float sA[2][BKR][BMR + 4];
    __shared__ __align__(16) float sB[2][BKR][BNR + 4];
    int64_t M = a.M, K = a.K;
    if (a.M_dev) {
        int64_t m = (int64_t)*a.M_dev;
        if (a.m_is_k) K = m < K ? m : K;
        else M = m < M ? m : M;
    }
    const int64_t i0 = (int64_t)blockIdx.y * BMR;
    const int j0 = blockIdx.x * BNR;
    if (i0 >= M) return;
    int64_t kb = 0, ke = K;
    if (EPI == kAtomic) {
        kb = (int64_t)blockIdx.z * a.k_chunk;
        ke = kb + a.k_chunk < K ? kb + a.k_chunk : K;
        if (kb >= ke) return;
    }
    const int tid = threadIdx.x, tx = tid & 7, ty = tid >> 3;
    const bool a_krow = a.sak == 1;
    const bool b_jrow = a.sbj == 1;
    float4 ra[A4], rb[B4];
    auto load_slice = [&](int64_t k0) {
#pragma unroll
        for (int q = 0; q < A4; q++) {
            const int idx = tid + q * NT;
            float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
            if (a_krow) {
                const int row = idx / (BKR / 4), k4 = (idx % (BKR / 4)) * 4;
                const int64_t gi = i0 + row, gk = k0 + k4;
                const float* src = a.A + gi * a.sai + gk;
                if (gi < M) {
                    if (gk + 3 < ke) v = *reinterpret_cast<const float4*>(src);
                    else {
                        if (gk + 0 < ke) v.x = src[0];
                        if (gk + 1 < ke) v.y = src[1];
                        if (gk + 2 < ke) v.z = src[2];
                    }
                }
            } else {
                const int k = idx / (BMR / 4), i4 = (idx % (BMR / 4)) * 4;
                const int64_t gi = i0 + i4, gk = k0 + k;
                const float* src = a.A + gi + gk * a.sak;
                if (gk < ke) {
                    if (gi + 3 < M) v = *reinterpret_cast<const float4*>(src);
                    else {
                        if (gi + 0 < M) v.x = src[0];
                        if (gi + 1 < M) v.y = src[1];
                        if (gi + 2 < M) v.z = src[2];
                    }
                }
            }
            ra[q] = v;
        }
#pragma unroll
        for (int q = 0; q < B4; q++) {
            const int idx = tid + q * NT;
            float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
            if (b_jrow) {
                const int k = idx / (BNR / 4), j4 = (idx % (BNR / 4)) * 4;
                const int64_t gk = k0 + k;
                if (gk < ke) v = *reinterpret_cast<const float4*>(a.B + gk * a.sbk + (j0 + j4));
            } else {
                const int j = idx / (BKR / 4), k4 = (idx % (BKR / 4)) * 4;
                const int64_t gk = k0 + k4;
                const float* src = a.B + (int64_t)(j0 + j) * a.sbj + gk;
                if (gk + 3 < ke) v = *reinterpret_cast<const float4*>(src);
                else {
                    if (gk + 0 < ke) v.x = src[0];
                    if (gk + 1 < ke) v.y = src[1];
                    if (gk + 2 < ke) v.z = src[2];
                }
            }
            rb[q] = v;
        }
    };
    auto store_slice = [&](int buf) {
#pragma unroll
        for (int q = 0; q < A4; q++) {
            const int idx = tid + q * NT;
            if (a_krow) {
                const int row = idx / (BKR / 4), k4 = (idx % (BKR / 4)) * 4;
                sA[buf][k4 + 0][row] = ra[q].x;
                sA[buf][k4 + 1][row] = ra[q].y;
                sA[buf][k4 + 2][row] = ra[q].z;
                sA[buf][k4 + 3][row] = ra[q].w;
            } else {
                const int k = idx / (BMR / 4), i4 = (idx % (BMR / 4)) * 4;
                *reinterpret_cast<float4*>(&sA[buf][k][i4]) = ra[q];
            }
        }
#pragma unroll
        for (int q = 0; q < B4; q++) {
            const int idx = tid + q * NT;
            if (b_jrow) {
                const int k = idx / (BNR / 4), j4 = (idx % (BNR / 4)) * 4;
                *reinterpret_cast<float4*>(&sB[buf][k][j4]) = rb[q];
            } else {
                const int j = idx / (BKR / 4), k4 = (idx % (BKR / 4)) * 4;
                sB[buf][k4 + 0][j] = rb[q].x;
                sB[buf][k4 + 1][j] = rb[q].y;
                sB[buf][k4 + 2][j] = rb[q].z;
                sB[buf][k4 + 3][j] = rb[q].w;
            }
        }
    };
    float acc[T8][T8];
#pragma unroll
    for (int r = 0; r < T8; r++)
#pragma unroll
        for (int c = 0; c < T8; c++) acc[r][c] = 0.f;
    load_slice(kb);
    store_slice(0);
    __syncthreads();
    int buf = 0;
    for (int64_t k0 = kb; k0 < ke; k0 += BKR) {
        const bool more = k0 + BKR < ke;
        if (more) load_slice(k0 + BKR);
#pragma unroll
        for (int kk = 0; kk < BKR; kk++) {
            const float4 a0 = *reinterpret_cast<const float4*>(&sA[buf][kk][ty * T8]);
            const float4 a1 = *reinterpret_cast<const float4*>(&sA[buf][kk][ty * T8 + 4]);
            const float4 b0 = *reinterpret_cast<const float4*>(&sB[buf][kk][tx * T8]);
            const float4 b1 = *reinterpret_cast<const float4*>(&sB[buf][kk][tx * T8 + 4]);
            const float av[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
            const float bv[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
            for (int r = 0; r < T8; r++)
#pragma unroll
                for (int c = 0; c < T8; c++) acc[r][c] += av[r] * bv[c];
        }
        if (more) {
            store_slice(buf ^ 1);
            __syncthreads();
            buf ^= 1;
        }
    }
#pragma unroll
    for (int r = 0; r < T8; r++) {
        const int64_t gi = i0 + ty * T8 + r;
        if (gi >= M) continue;
        const int gj = j0 + tx * T8;
        float* dst = a.C + gi * a.ldc + gj;
        if (EPI == kAtomic) {
#pragma unroll
            for (int c = 0; c < T8; c++) atomicAdd(dst + c, acc[r][c]);
        } else {
#pragma unroll
        for (int h4 = 0; h4 < 2; h4++) {
            float4 v = make_float4(acc[r][4 * h4], acc[r][4 * h4 + 1], acc[r][4 * h4 + 2], acc[r][4 * h4 + 3]);
            if (EPI == kRelu) {
                v.x = fmaxf(v.x, 0.f); v.y = fmaxf(v.y, 0.f); v.z = fmaxf(v.z, 0.f); v.w = fmaxf(v.w, 0.f);
            } else if (EPI == kMask) {
                float4 m = *reinterpret_cast<const float4*>(a.mask + gi * a.ldc + gj + 4 * h4);
                v.x = m.x > 0.f ? v.x : 0.f; v.y = m.y > 0.f ? v.y : 0.f;
                v.z = m.z > 0.f ? v.z : 0.f; v.w = m.w > 0.f ? v.w : 0.f;
            }
            *reinterpret_cast<float4*>(dst + 4 * h4) = v;
        }
        }
    }
}

static bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15) == 0; }

template <int EPI>
nif_status gemm(nif_handle* h, GemmArgs a, cudaStream_t s, int splits = 1) {
    // the register-blocked kernel serves aligned shapes with N % 64 == 0 and K-slices of 16
    bool big = a.N % 64 == 0 && (a.sak == 1 || a.sai == 1) && (a.sbj == 1 || a.sbk == 1) && aligned16(a.A) &&
               aligned16(a.B) && aligned16(a.C) && a.ldc % 4 == 0 && (a.sak == 1 ? a.sai % 4 == 0 : a.sak % 4 == 0) &&
               (a.sbj == 1 ? a.sbk % 4 == 0 : a.sbj % 4 == 0) && (!a.mask || aligned16(a.mask)) &&
               (a.m_is_k || a.K % 16 == 0);
    // 128-row tiles for long reductions over many rows, 64-row tiles otherwise (more resident blocks)
    const bool tall = big && a.M >= 96 && !a.m_is_k && (a.K > 64 || a.N >= 512);
    const int bm = big ? (tall ? 128 : 64) : BM;
    const int64_t tiles = (int64_t)((a.N + 63) / 64) * ((a.M + bm - 1) / bm);
    auto split_rows = [&](int64_t waves_sms) {
        int64_t want = std::max<int64_t>(1, (waves_sms + tiles - 1) / tiles);
        int64_t chunk = (a.K + want - 1) / want;
        return std::max<int64_t>(256, (chunk + 15) / 16 * 16);
    };
    // split the row reduction so that the grid covers the GPU about four times
    if (EPI == kAtomic) a.k_chunk = split_rows(4 * (int64_t)h->num_sms);
    // the 8x8-per-thread kernel pays off when each block reduces over >= 512
    // (it holds fewer warps per SM; short reductions are prologue-bound)
    const bool rt = big && ((EPI == kAtomic ? a.k_chunk : a.K) >= 512 || (tall && a.N >= 512));
    if (EPI == kAtomic) {
        if (rt) a.k_chunk = std::max<int64_t>(512, split_rows(8 * (int64_t)h->num_sms));
        splits = (int)((a.K + a.k_chunk - 1) / a.k_chunk);
    }
    if (rt && tall) {
        dim3 grid(a.N / 64, (unsigned)((a.M + 127) / 128), splits);
        k_sgemm_rt<EPI, 128><<<grid, 128, 0, s>>>(a);
    } else if (rt) {
        dim3 grid(a.N / 64, (unsigned)((a.M + 63) / 64), splits);
        k_sgemm_rt<EPI, 64><<<grid, 64, 0, s>>>(a);
    } else if (big && tall) {
        dim3 grid(a.N / 64, (unsigned)((a.M + 127) / 128), splits);
        k_sgemm_big<EPI, 128><<<grid, 256, 0, s>>>(a);
    } else if (big) {
        dim3 grid(a.N / 64, (unsigned)((a.M + 63) / 64), splits);
        k_sgemm_big<EPI, 64><<<grid, 256, 0, s>>>(a);
    } else {
        dim3 grid((a.N + BN - 1) / BN, (unsigned)((a.M + BM - 1) / BM), splits);
        k_sgemm<EPI><<<grid, 256, 0, s>>>(a);
    }
    NIF_CK_LAUNCH(h);
    return NIF_OK;
}

}  // namespace

nif_status nif_mlp_fwd_fp32_run(nif_handle* h, const float* x, const uint32_t* n_dev, int64_t n_max, float* out,
                                float* acts, cudaStream_t s) {
    NifProf prof_(h, "mlp_fwd_fp32", s);
    if (n_max <= 0) return NIF_OK;
    const float* in = x;
    int64_t in_ld = h->in_dim;
    for (int l = 0; l < h->n_layers; l++) {
        bool last = l == h->n_layers - 1;
        GemmArgs a{};
        a.A = in; a.sai = in_ld; a.sak = 1;
        a.B = h->d_params + h->off_layer[l]; a.sbk = 1; a.sbj = h->lay_in[l];
        a.M = n_max; a.N = h->lay_out[l]; a.K = h->lay_in[l];
        a.M_dev = n_dev; a.m_is_k = 0;
        if (last) {
            a.C = out; a.ldc = NIF_OUT;
            nif_status st = gemm<kStore>(h, a, s);
            if (st != NIF_OK) return st;
        } else {
            float* dst = acts + (int64_t)l * n_max * h->W;
            a.C = dst; a.ldc = h->W;
            nif_status st = gemm<kRelu>(h, a, s);
            if (st != NIF_OK) return st;
            in = dst;
            in_ld = h->W;
        }
    }
    return NIF_OK;
}

nif_status nif_mlp_bwd_fp32_run(nif_handle* h, const float* x, const uint32_t* n_dev, int64_t n_max,
                                const float* acts, const float* dout, float* dx, cudaStream_t s, bool want_dw,
                                cudaStream_t aux) {
    NifProf prof_(h, "mlp_bwd_fp32", s);
    if (n_max <= 0) return NIF_OK;
    nif_status st = nif_grow(h, h->b_dout, sizeof(float) * (size_t)n_max * h->W * 2);
    if (st != NIF_OK) return st;
    float* gbuf[2] = {(float*)h->b_dout.p, (float*)h->b_dout.p + (size_t)n_max * h->W};
    const float* g = dout;
    int64_t g_ld = NIF_OUT;
    int cur = 0;
    for (int l = h->n_layers - 1; l >= 0; l--) {
        const float* in = l == 0 ? x : acts + (int64_t)(l - 1) * n_max * h->W;
        int64_t in_ld = l == 0 ? h->in_dim : h->W;
        int nout = h->lay_out[l], nin = h->lay_in[l];
        // dW_l += g^T in : C [nout x nin], reduction over rows
        GemmArgs w{};
        w.A = g; w.sai = 1; w.sak = g_ld;
        w.B = in; w.sbk = in_ld; w.sbj = 1;
        w.C = h->d_grad + h->off_layer[l]; w.ldc = nin;
        w.M = nout; w.N = nin; w.K = n_max; w.M_dev = n_dev; w.m_is_k = 1; w.k_chunk = 0;
        if (want_dw && l == 0 && aux) {
            // dY_0 is final: the layer-0 weight gradient overlaps dX_0 and what follows
            NIF_CK(h, cudaEventRecord(h->ev_fork, s));
            NIF_CK(h, cudaStreamWaitEvent(aux, h->ev_fork, 0));
            {
                NifProf prof_dw(h, "mlp_dw0_fp32", aux);
                if ((st = gemm<kAtomic>(h, w, aux)) != NIF_OK) return st;
            }
            NIF_CK(h, cudaEventRecord(h->ev_join, aux));
        } else if (want_dw && (st = gemm<kAtomic>(h, w, s)) != NIF_OK) {
            return st;
        }
        // d(in) = g W_l : [n x nin], masked by the ReLU of the layer below
        if (l == 0 && !dx) break;
        GemmArgs d{};
        d.A = g; d.sai = g_ld; d.sak = 1;
        d.B = h->d_params + h->off_layer[l]; d.sbk = nin; d.sbj = 1;
        d.M = n_max; d.N = nin; d.K = nout; d.M_dev = n_dev; d.m_is_k = 0;
        if (l == 0) {
            d.C = dx; d.ldc = h->in_dim;
            st = gemm<kStore>(h, d, s);
        } else {
            d.C = gbuf[cur]; d.ldc = h->W; d.mask = in;
            st = gemm<kMask>(h, d, s);
            g = gbuf[cur];
            g_ld = h->W;
            cur ^= 1;
        }
        if (st != NIF_OK) return st;
    }
    return NIF_OK;
}
