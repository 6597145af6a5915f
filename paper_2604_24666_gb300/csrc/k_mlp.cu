// k_mlp.cu -- FP32 (FFMA) path of the MLP (Sec. 2, Fig. 2d): H hidden ReLU
// layers without bias and a linear output layer, forward and backward.
//
// All products are one tiled SGEMM kernel C = A * B with arbitrary element
// strides (so the same kernel serves X W^T, dY W and dY^T X), 64x64 output
// tiles, 16-deep K slices staged in shared memory, 4x4 outputs per thread,
// and an epilogue chosen per call: store, ReLU, ReLU-derivative mask, or
// split-K atomic accumulation (for weight gradients summed over rows).
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

template <int EPI>
nif_status gemm(nif_handle* h, GemmArgs a, cudaStream_t s, int splits = 1) {
    dim3 grid((a.N + BN - 1) / BN, (unsigned)((a.M + BM - 1) / BM), splits);
    k_sgemm<EPI><<<grid, 256, 0, s>>>(a);
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
                                const float* acts, const float* dout, float* dx, cudaStream_t s) {
    NifProf prof_(h, "mlp_bwd_fp32", s);
    if (n_max <= 0) return NIF_OK;
    nif_status st = nif_grow(h, h->b_dout, sizeof(float) * (size_t)n_max * h->W * 2);
    if (st != NIF_OK) return st;
    float* gbuf[2] = {(float*)h->b_dout.p, (float*)h->b_dout.p + (size_t)n_max * h->W};
    const float* g = dout;
    int64_t g_ld = NIF_OUT;
    int cur = 0;
    const int64_t chunk = 4096;
    int splits = (int)((n_max + chunk - 1) / chunk);
    for (int l = h->n_layers - 1; l >= 0; l--) {
        const float* in = l == 0 ? x : acts + (int64_t)(l - 1) * n_max * h->W;
        int64_t in_ld = l == 0 ? h->in_dim : h->W;
        int nout = h->lay_out[l], nin = h->lay_in[l];
        // dW_l += g^T in : C [nout x nin], reduction over rows
        GemmArgs w{};
        w.A = g; w.sai = 1; w.sak = g_ld;
        w.B = in; w.sbk = in_ld; w.sbj = 1;
        w.C = h->d_grad + h->off_layer[l]; w.ldc = nin;
        w.M = nout; w.N = nin; w.K = n_max; w.M_dev = n_dev; w.m_is_k = 1; w.k_chunk = chunk;
        st = gemm<kAtomic>(h, w, s, splits);
        if (st != NIF_OK) return st;
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
