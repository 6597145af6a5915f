// k_probe.cu -- measured ceilings of the memory patterns the encoding kernels
// are bound by (diagnostics; the paper has no counterpart): random 8- and
// 16-byte FP32 reductions into a table-gradient-sized buffer held in L2 (the
// encoding backward's red.global.add.v2/.v4.f32), and random 8- and 4-byte
// row loads from a table (the encoding forward's FP32 float2 / FP16 half2
// corner gathers). Every thread draws rows from its own xorshift stream;
// each iteration issues kInFlight independent accesses so that throughput,
// not latency, is measured. The warp-coalesced variants draw one row block
// per warp (its 32 lanes touch 32 consecutive rows, whole 32-byte sectors):
// the fully random ones measure the L2's rate for scattered accesses (one
// sector per lane), the coalesced ones its rate when every sector is used.
#include <algorithm>

#include "nif_internal.cuh"

namespace {

constexpr int kInFlight = 8;

__device__ __forceinline__ uint32_t xorshift(uint32_t& s) {
    s ^= s << 13;
    s ^= s >> 17;
    s ^= s << 5;
    return s;
}

__device__ __forceinline__ uint32_t seed_of(uint32_t tid, uint32_t salt) {
    uint32_t s = tid * 2654435761u ^ (salt * 0x9E3779B9u + 0x7F4A7C15u);
    return s ? s : 1u;
}

// rows: 8-byte rows in the buffer (power of two); vec4: 16-byte reductions of
// two adjacent rows (row index even)
template <bool kVec4, bool kWarp>
__global__ void __launch_bounds__(256) k_probe_red(float* __restrict__ buf, uint32_t rows, int iters, uint32_t salt) {
    const uint32_t lane = threadIdx.x & 31u;
    uint32_t s = seed_of(kWarp ? (blockIdx.x * blockDim.x + threadIdx.x) >> 5 : blockIdx.x * blockDim.x + threadIdx.x,
                         salt);
    const uint32_t mask = rows - 1u;
    for (int it = 0; it < iters; it++) {
#pragma unroll
        for (int q = 0; q < kInFlight; q++) {
            uint32_t r = xorshift(s) & mask;
            if (kWarp) r = (r & ~(kVec4 ? 63u : 31u)) + (kVec4 ? 2u : 1u) * lane;
            if (kVec4) {
                r &= ~1u;
                asm volatile("red.global.add.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(buf + 2 * (size_t)r), "f"(1e-30f),
                             "f"(1e-30f), "f"(1e-30f), "f"(1e-30f)
                             : "memory");
            } else {
                asm volatile("red.global.add.v2.f32 [%0], {%1, %2};" ::"l"(buf + 2 * (size_t)r), "f"(1e-30f),
                             "f"(1e-30f)
                             : "memory");
            }
        }
    }
}

// random row loads: 8-byte rows (float2) or 4-byte rows (half2); the sum goes
// to sink[thread] so the loads cannot be dropped
template <bool kHalf, bool kWarp>
__global__ void __launch_bounds__(256) k_probe_load(const void* __restrict__ tab, uint32_t rows, int iters,
                                                    uint32_t salt, float* __restrict__ sink) {
    const uint32_t lane = threadIdx.x & 31u;
    uint32_t s = seed_of(kWarp ? (blockIdx.x * blockDim.x + threadIdx.x) >> 5 : blockIdx.x * blockDim.x + threadIdx.x,
                         salt);
    const uint32_t mask = rows - 1u;
    float acc = 0.f;
    for (int it = 0; it < iters; it++) {
        float v[kInFlight];
#pragma unroll
        for (int q = 0; q < kInFlight; q++) {
            uint32_t r = xorshift(s) & mask;
            if (kWarp) r = (r & ~31u) + lane;
            if (kHalf) {
                const __half2 h = __ldg(reinterpret_cast<const __half2*>(tab) + r);
                v[q] = __low2float(h) + __high2float(h);
            } else {
                const float2 f = __ldg(reinterpret_cast<const float2*>(tab) + r);
                v[q] = f.x + f.y;
            }
        }
#pragma unroll
        for (int q = 0; q < kInFlight; q++) acc += v[q];
    }
    sink[blockIdx.x * blockDim.x + threadIdx.x] = acc;
}

}  // namespace

extern "C" nif_status nif_probe_memory(nif_handle* h, int kind, void* buf, size_t bytes, int iters, double* gbs,
                                       double* ms_out, void* stream) {
    if (!h) return NIF_ERR_ARG;
    const bool warp = kind >= NIF_PROBE_RED8_WARP;
    const int base = warp ? kind - NIF_PROBE_RED8_WARP + NIF_PROBE_RED8 : kind;
    const size_t row = base == NIF_PROBE_LOAD4 ? 4 : 8;
    const size_t rows = bytes / row;
    if (!buf || rows < 1024 || (rows & (rows - 1)) || rows > (1ull << 31) || iters < 1 || iters > (1 << 20) ||
        (reinterpret_cast<uintptr_t>(buf) & 15) ||
        kind < NIF_PROBE_RED8 || kind > NIF_PROBE_LOAD4_WARP)
        return nif_fail(h, NIF_ERR_ARG, "probe: kind, 16-byte aligned buffer of a power-of-two row count >= 1024, iters");
    cudaStream_t s = (cudaStream_t)stream;
    const int threads = 256;
    const int blocks = h->num_sms * 8;              // 2048 threads per SM
    const size_t n_thr = (size_t)threads * blocks;
    float* sink = nullptr;
    if (base == NIF_PROBE_LOAD8 || base == NIF_PROBE_LOAD4) {
        nif_status st = nif_grow(h, h->b_scan, sizeof(float) * n_thr);
        if (st != NIF_OK) return st;
        sink = (float*)h->b_scan.p;
    }
    auto launch = [&](uint32_t salt) -> nif_status {
        const uint32_t nr = (uint32_t)rows;
        switch (kind) {
            case NIF_PROBE_RED8: k_probe_red<false, false><<<blocks, threads, 0, s>>>((float*)buf, nr, iters, salt); break;
            case NIF_PROBE_RED16: k_probe_red<true, false><<<blocks, threads, 0, s>>>((float*)buf, nr, iters, salt); break;
            case NIF_PROBE_LOAD8: k_probe_load<false, false><<<blocks, threads, 0, s>>>(buf, nr, iters, salt, sink); break;
            case NIF_PROBE_LOAD4: k_probe_load<true, false><<<blocks, threads, 0, s>>>(buf, nr, iters, salt, sink); break;
            case NIF_PROBE_RED8_WARP: k_probe_red<false, true><<<blocks, threads, 0, s>>>((float*)buf, nr, iters, salt); break;
            case NIF_PROBE_RED16_WARP: k_probe_red<true, true><<<blocks, threads, 0, s>>>((float*)buf, nr, iters, salt); break;
            case NIF_PROBE_LOAD8_WARP: k_probe_load<false, true><<<blocks, threads, 0, s>>>(buf, nr, iters, salt, sink); break;
            default: k_probe_load<true, true><<<blocks, threads, 0, s>>>(buf, nr, iters, salt, sink); break;
        }
        NIF_CK_LAUNCH(h);
        return NIF_OK;
    };
    cudaEvent_t a, b;
    NIF_CK(h, cudaEventCreate(&a));
    NIF_CK(h, cudaEventCreate(&b));
    nif_status st = launch(1);                      // brings the buffer into L2
    const int reps = 5;
    if (st == NIF_OK) {
        NIF_CK(h, cudaEventRecord(a, s));
        for (int r = 0; r < reps && st == NIF_OK; r++) st = launch(2 + r);
        NIF_CK(h, cudaEventRecord(b, s));
        NIF_CK(h, cudaEventSynchronize(b));
    }
    float ms = 0.f;
    if (st == NIF_OK) NIF_CK(h, cudaEventElapsedTime(&ms, a, b));
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    if (st != NIF_OK) return st;
    const double per = (double)ms / reps;
    const double payload = base == NIF_PROBE_RED16 ? 16.0 : (base == NIF_PROBE_LOAD4 ? 4.0 : 8.0);
    const double total = payload * (double)n_thr * (double)iters * kInFlight;
    if (gbs) *gbs = total / (per * 1e-3) / 1e9;
    if (ms_out) *ms_out = per;
    return NIF_OK;
}

extern "C" nif_status nif_encoder_points(nif_handle* h, int64_t* n_points, int64_t* n_segments) {
    if (!h) return NIF_ERR_ARG;
    const nif_handle::PointList& pl = h->enc_points;
    if (!pl.pts || !pl.n_pts) return nif_fail(h, NIF_ERR_STATE, "no segment encoding has listed its end points yet");
    uint32_t np = 0, ns = 0;
    NIF_CK(h, cudaDeviceSynchronize());
    NIF_CK(h, cudaMemcpy(&np, pl.n_pts, sizeof(uint32_t), cudaMemcpyDeviceToHost));
    if (pl.n_dev) NIF_CK(h, cudaMemcpy(&ns, pl.n_dev, sizeof(uint32_t), cudaMemcpyDeviceToHost));
    else ns = (uint32_t)pl.n_max;
    if (n_points) *n_points = np;
    if (n_segments) *n_segments = std::min<int64_t>(ns, pl.n_max);
    return NIF_OK;
}
