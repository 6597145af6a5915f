// k_encode.cu -- hybrid encoding psi = phi o gamma (Eq. 1) forward and
// backward.
//
// gamma(x) = [x, sin(2^k x), cos(2^k x)]_{k<F} gives P = 1 + 2F 3-vectors;
// each goes through the same multiresolution grid phi (Sec. 2.3: "each ...
// frequency-modulated sample is independently processed by the multi-level
// hash grid encoder") at u = x (x term) or u = (g + 1)/2 (sin and cos terms).
// Level l has N_l cells per axis: q = fl32(u * N_l), i0 = min(floor(q), N_l-1),
// w = q - i0; the row of grid vertex (i,j,k) is the dense index
// i + j(N_l+1) + k(N_l+1)^2 when (N_l+1)^3 <= T and otherwise the spatial hash
// (i * 1 ^ j * 2654435761 ^ k * 805459861) mod T of Mueller et al. (2022).
//
// One thread owns one (point, term) pair: it evaluates the term's sines once
// and loops over the L levels, issuing the 8 corner loads of a level
// back-to-back (float2 = both features of an FP32 row, half2 of an FP16 row).
#include <algorithm>

#include "enc_grid.cuh"
#include "nif_internal.cuh"

namespace {

__device__ __forceinline__ uint32_t grid_row(uint32_t i, uint32_t j, uint32_t k, int Nl, bool dense,
                                             uint32_t T) {
    if (dense) {
        uint32_t s = (uint32_t)Nl + 1u;
        return i + j * s + k * s * s;
    }
    return (i ^ (j * 2654435761u) ^ (k * 805459861u)) & (T - 1u);
}

// du/dp of term t (diagonal), zero where p was clamped
__device__ __forceinline__ float3 term_dudp(float3 p, int t) {
    if (t == 0) return make_float3(1.f, 1.f, 1.f);
    int k = (t - 1) >> 1;
    float f = (float)(1 << k);
    float sx, cx, sy, cy, sz, cz;
    sincosf(f * p.x, &sx, &cx);
    sincosf(f * p.y, &sy, &cy);
    sincosf(f * p.z, &sz, &cz);
    if ((t - 1) & 1) return make_float3(-0.5f * f * sx, -0.5f * f * sy, -0.5f * f * sz);
    return make_float3(0.5f * f * cx, 0.5f * f * cy, 0.5f * f * cz);
}

template <typename TT>
__device__ __forceinline__ float2 load_row(const TT* tab, uint32_t row);
template <>
__device__ __forceinline__ float2 load_row<float>(const float* tab, uint32_t row) {
    return __ldg(reinterpret_cast<const float2*>(tab) + row);
}
template <>
__device__ __forceinline__ float2 load_row<__half>(const __half* tab, uint32_t row) {
    __half2 v = __ldg(reinterpret_cast<const __half2*>(tab) + row);
    return __half22float2(v);
}

template <typename OT>
__device__ __forceinline__ void store2(OT* out, int64_t i, float2 v);
template <>
__device__ __forceinline__ void store2<float>(float* out, int64_t i, float2 v) {
    *reinterpret_cast<float2*>(out + i) = v;
}
template <>
__device__ __forceinline__ void store2<__nv_bfloat16>(__nv_bfloat16* out, int64_t i, float2 v) {
    *reinterpret_cast<__nv_bfloat162*>(out + i) = __floats2bfloat162_rn(v.x, v.y);
}
template <>
__device__ __forceinline__ void store2<__half>(__half* out, int64_t i, float2 v) {
    *reinterpret_cast<__half2*>(out + i) = __floats2half2_rn(v.x, v.y);
}

// phi at u for all levels: writes L float2 starting at out[o]
template <typename TT, typename OT>
__device__ __forceinline__ void grid_all_levels(const GridInfo& g, const TT* __restrict__ tab, float3 u,
                                                OT* __restrict__ out, int64_t o, int32_t* rows,
                                                int64_t ro) {
    for (int l = 0; l < g.L; l++) {
        int Nl = g.res[l];
        bool dense = (g.dense_mask >> l) & 1u;
        Cell c = cell_of(u, Nl);
        const TT* tl = tab + (int64_t)l * g.T * 2;
        float2 acc = make_float2(0.f, 0.f);
        float2 v[8];
#pragma unroll
        for (int q = 0; q < 8; q++)
            v[q] = load_row<TT>(tl, grid_row(c.ix + (q & 1), c.iy + ((q >> 1) & 1), c.iz + ((q >> 2) & 1), Nl,
                                             dense, g.T));
#pragma unroll
        for (int q = 0; q < 8; q++) {
            float w = ((q & 1) ? c.wx : 1.f - c.wx) * ((q & 2) ? c.wy : 1.f - c.wy) * ((q & 4) ? c.wz : 1.f - c.wz);
            acc.x += w * v[q].x;
            acc.y += w * v[q].y;
        }
        store2<OT>(out, o + 2 * l, acc);
        if (rows) rows[ro + l] = (int32_t)grid_row(c.ix, c.iy, c.iz, Nl, dense, g.T);
    }
}

template <typename TT, typename OT>
__global__ void __launch_bounds__(256) k_encode_points(GridInfo g, const TT* __restrict__ tab,
                                                       const float* __restrict__ pts, int64_t n,
                                                       OT* __restrict__ out, int32_t* __restrict__ rows) {
    int64_t gid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (gid >= n * g.P) return;
    int64_t i = gid / g.P;
    int t = (int)(gid - i * g.P);
    float3 p = clamp01(make_float3(pts[3 * i], pts[3 * i + 1], pts[3 * i + 2]));
    float3 u = term_u(p, t);
    grid_all_levels<TT, OT>(g, tab, u, out, gid * g.L * 2, rows, gid * g.L);
}

// Forward over segments, all levels of one (segment, endpoint, term) in
// registers: corner rows from one base index (dense) or three partial hashes,
// weights from the x-y products, and the L feature pairs written with 16-byte
// stores at the end (LMAX >= L, compile-time for full unrolling).
template <typename OT>
struct OutPair;
template <>
struct OutPair<float> {
    using T = float2;
    static __device__ __forceinline__ T make(float a, float b) { return make_float2(a, b); }
};
template <>
struct OutPair<__nv_bfloat16> {
    using T = __nv_bfloat162;
    static __device__ __forceinline__ T make(float a, float b) { return __floats2bfloat162_rn(a, b); }
};
template <>
struct OutPair<__half> {
    using T = __half2;
    static __device__ __forceinline__ T make(float a, float b) { return __floats2half2_rn(a, b); }
};

// Along a ray the exit point of a voxel is, bit for bit, the entry point of
// the next one where the two share a face (the same hull triangle in the same
// vertex order gives the same t; the same inverse gives the same rest point):
// about two thirds of the segments of the synthetic workloads. k_dup_flags
// marks them (u = 1: p0 repeats the previous p1, u = 2: both end points are
// new, u = 0: past the live count), a scan of u numbers the distinct points,
// k_point_list lists them as 2 s + e, and the encoder runs once per distinct
// point, writing a repeated point's features into both rows.
__global__ void __launch_bounds__(256) k_dup_flags(const nif_linseg* __restrict__ lin,
                                                   const uint32_t* __restrict__ n_dev, int64_t n_max,
                                                   uint32_t* __restrict__ u) {
    int64_t n = n_dev ? (int64_t)*n_dev : n_max;
    if (n > n_max) n = n_max;
    for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < n_max;
         s += (int64_t)gridDim.x * blockDim.x) {
        uint32_t v = 0;
        if (s < n) {
            v = 2;
            if (s > 0) {
                const float* a = reinterpret_cast<const float*>(lin + s);
                const float* b = reinterpret_cast<const float*>(lin + s - 1) + 3;
                if (a[0] == b[0] && a[1] == b[1] && a[2] == b[2]) v = 1;
            }
        }
        u[s] = v;
    }
}

__global__ void __launch_bounds__(256) k_point_list(const uint32_t* __restrict__ u, const uint32_t* __restrict__ off,
                                                    int64_t n_max, uint32_t* __restrict__ pts) {
    for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < n_max;
         s += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t v = u[s], o = off[s];
        if (v == 2) {
            pts[o] = (uint32_t)(2 * s);
            pts[o + 1] = (uint32_t)(2 * s + 1);
        } else if (v == 1) {
            pts[o] = (uint32_t)(2 * s + 1);
        }
    }
}

// pts (nullable): the distinct points (2 s + e, *n_pts_dev of them) and dupf
// the flags of k_dup_flags; without them every (segment, end point) is encoded
template <typename TT, typename OT, int LMAX>
__global__ void __launch_bounds__(512) k_encode_segments_v(GridInfo g, const TT* __restrict__ tab,
                                                           const nif_linseg* __restrict__ lin,
                                                           const uint32_t* __restrict__ n_dev, int64_t n_max,
                                                           OT* __restrict__ out, const uint32_t* __restrict__ pts,
                                                           const uint32_t* __restrict__ n_pts_dev,
                                                           const uint32_t* __restrict__ dupf) {
    using P2 = typename OutPair<OT>::T;
    int64_t n = n_dev ? (int64_t)*n_dev : n_max;
    if (n > n_max) n = n_max;
    const int64_t n_points = pts ? (int64_t)*n_pts_dev : 2 * n;
    // a warp takes one gamma term of 32 consecutive points: points along a ray
    // fall in the same coarse cells, so their corner loads merge into fewer
    // L1 wavefronts than 32 lanes spread over every term of a few points
    const int64_t n_work = (n_points + 31) / 32 * 32 * g.P;
    for (int64_t gid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; gid < n_work;
         gid += (int64_t)gridDim.x * blockDim.x) {
        const int64_t grp = gid >> 5;
        const int t = (int)(grp % g.P);
        const int64_t k = (grp / g.P) * 32 + (gid & 31);
        if (k >= n_points) continue;
        const int64_t pt = pts ? (int64_t)pts[k] : k;
        const int64_t s = pt >> 1;
        const int e = (int)(pt & 1);
        const float* L = reinterpret_cast<const float*>(lin + s) + 3 * e;
        float3 u = term_u(clamp01(make_float3(L[0], L[1], L[2])), t);
        P2 res[LMAX];
#pragma unroll
        for (int l = 0; l < LMAX; l++) {
            if (l >= g.L) break;
            const Cell c = cell_of(u, g.res[l]);
            typename RawRow<TT>::T vr[8];
            level_gather<TT>(g, tab, l, c, vr);
            const float wx1 = c.wx, wx0 = 1.f - c.wx, wy1 = c.wy, wy0 = 1.f - c.wy;
            const float wz1 = c.wz, wz0 = 1.f - c.wz;
            const float wxy[4] = {wx0 * wy0, wx1 * wy0, wx0 * wy1, wx1 * wy1};
            float2 acc = make_float2(0.f, 0.f);
#pragma unroll
            for (int q = 0; q < 8; q++) {
                const float w = wxy[q & 3] * ((q & 4) ? wz1 : wz0);
                const float2 v = RawRow<TT>::f2(vr[q]);
                acc.x += w * v.x;
                acc.y += w * v.y;
            }
            res[l] = OutPair<OT>::make(acc.x, acc.y);
        }
        // the row of (s, e, t), and of (s + 1, 0, t) when that end point repeats this one
        const bool twice = pts && e == 1 && s + 1 < n_max && dupf[s + 1] == 1;
        P2* o = reinterpret_cast<P2*>(out + ((s * 2 + e) * g.P + t) * g.L * 2);
        P2* o2 = reinterpret_cast<P2*>(out + ((s + 1) * 2 * g.P + t) * g.L * 2);
        constexpr int per16 = 16 / sizeof(P2);           // pairs per 16-byte store
        if ((g.L % per16) == 0) {
#pragma unroll
            for (int l = 0; l < LMAX; l += per16) {
                if (l >= g.L) break;
                uint4 w4;
                uint32_t* w = reinterpret_cast<uint32_t*>(&w4);
#pragma unroll
                for (int kk = 0; kk < per16; kk++) {
                    const uint32_t* src = reinterpret_cast<const uint32_t*>(&res[l + kk]);
#pragma unroll
                    for (int q = 0; q < (int)(sizeof(P2) / 4); q++) w[kk * (sizeof(P2) / 4) + q] = src[q];
                }
                *reinterpret_cast<uint4*>(o + l) = w4;
                if (twice) *reinterpret_cast<uint4*>(o2 + l) = w4;
            }
        } else {
#pragma unroll
            for (int l = 0; l < LMAX; l++) {
                if (l >= g.L) break;
                o[l] = res[l];
                if (twice) o2[l] = res[l];
            }
        }
    }
}

template <typename TT, typename OT>
__global__ void __launch_bounds__(512) k_encode_segments(GridInfo g, const TT* __restrict__ tab,
                                                         const nif_linseg* __restrict__ lin,
                                                         const uint32_t* __restrict__ n_dev, int64_t n_max,
                                                         OT* __restrict__ out) {
    int64_t n = n_dev ? (int64_t)*n_dev : n_max;
    if (n > n_max) n = n_max;
    int per = 2 * g.P;
    for (int64_t gid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; gid < n * per;
         gid += (int64_t)gridDim.x * blockDim.x) {
        int64_t s = gid / per;
        int r = (int)(gid - s * per);
        int e = r >= g.P;
        int t = r - e * g.P;
        const float* L = reinterpret_cast<const float*>(lin + s) + 3 * e;
        float3 p = clamp01(make_float3(L[0], L[1], L[2]));
        float3 u = term_u(p, t);
        grid_all_levels<TT, OT>(g, tab, u, out, gid * g.L * 2, nullptr, 0);
    }
}

// backward: scatter w * dfeat into the FP32 table gradient; optional d/dp
__device__ __forceinline__ void grid_backward(const GridInfo& g, const float* __restrict__ tab, float3 u,
                                              const float* __restrict__ df, float* __restrict__ dtab,
                                              float3* du) {
    float3 acc = make_float3(0.f, 0.f, 0.f);
    for (int l = 0; l < g.L; l++) {
        int Nl = g.res[l];
        bool dense = (g.dense_mask >> l) & 1u;
        Cell c = cell_of(u, Nl);
        float2 gr = *reinterpret_cast<const float2*>(df + 2 * l);
        float* dl = dtab + (int64_t)l * g.T * 2;
        const float* tl = tab + (int64_t)l * g.T * 2;
        float3 dl_du = make_float3(0.f, 0.f, 0.f);
#pragma unroll
        for (int q = 0; q < 8; q++) {
            uint32_t row = grid_row(c.ix + (q & 1), c.iy + ((q >> 1) & 1), c.iz + ((q >> 2) & 1), Nl, dense, g.T);
            float fx = (q & 1) ? c.wx : 1.f - c.wx;
            float fy = (q & 2) ? c.wy : 1.f - c.wy;
            float fz = (q & 4) ? c.wz : 1.f - c.wz;
            float w = fx * fy * fz;
            atomicAdd(reinterpret_cast<float2*>(dl) + row, make_float2(w * gr.x, w * gr.y));
            if (du) {
                float2 v = __ldg(reinterpret_cast<const float2*>(tl) + row);
                float val = v.x * gr.x + v.y * gr.y;
                dl_du.x += ((q & 1) ? 1.f : -1.f) * fy * fz * val;
                dl_du.y += ((q & 2) ? 1.f : -1.f) * fx * fz * val;
                dl_du.z += ((q & 4) ? 1.f : -1.f) * fx * fy * val;
            }
        }
        float fn = (float)Nl;
        acc.x += fn * dl_du.x;
        acc.y += fn * dl_du.y;
        acc.z += fn * dl_du.z;
    }
    if (du) *du = acc;
}

__global__ void __launch_bounds__(256) k_encode_points_bwd(GridInfo g, const float* __restrict__ tab,
                                                           const float* __restrict__ pts, int64_t n,
                                                           const float* __restrict__ dfeats,
                                                           float* __restrict__ dtab, float* __restrict__ dpts) {
    int64_t gid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (gid >= n * g.P) return;
    int64_t i = gid / g.P;
    int t = (int)(gid - i * g.P);
    float3 raw = make_float3(pts[3 * i], pts[3 * i + 1], pts[3 * i + 2]);
    float3 p = clamp01(raw);
    float3 u = term_u(p, t);
    float3 du;
    grid_backward(g, tab, u, dfeats + gid * g.L * 2, dtab, dpts ? &du : nullptr);
    if (dpts) {
        float3 j = term_dudp(p, t);
        if (raw.x < 0.f || raw.x > 1.f) j.x = 0.f;
        if (raw.y < 0.f || raw.y > 1.f) j.y = 0.f;
        if (raw.z < 0.f || raw.z > 1.f) j.z = 0.f;
        atomicAdd(dpts + 3 * i, du.x * j.x);
        atomicAdd(dpts + 3 * i + 1, du.y * j.y);
        atomicAdd(dpts + 3 * i + 2, du.z * j.z);
    }
}

__global__ void __launch_bounds__(256) k_encode_segments_bwd(GridInfo g, const float* __restrict__ tab,
                                                             const nif_linseg* __restrict__ lin,
                                                             const uint32_t* __restrict__ n_dev, int64_t n_max,
                                                             const float* __restrict__ dfeats,
                                                             float* __restrict__ dtab) {
    int64_t n = n_dev ? (int64_t)*n_dev : n_max;
    if (n > n_max) n = n_max;
    int per = 2 * g.P;
    for (int64_t gid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; gid < n * per;
         gid += (int64_t)gridDim.x * blockDim.x) {
        int64_t s = gid / per;
        int r = (int)(gid - s * per);
        int e = r >= g.P;
        int t = r - e * g.P;
        const float* L = reinterpret_cast<const float*>(lin + s) + 3 * e;
        float3 p = clamp01(make_float3(L[0], L[1], L[2]));
        float3 u = term_u(p, t);
        grid_backward(g, tab, u, dfeats + gid * g.L * 2, dtab, nullptr);
    }
}

// Backward with the dense coarse levels 0..Lc-1 accumulated in shared memory
// by each persistent block and flushed once; finer levels use global float2
// reductions. soff[l] is the float offset of level l's block in shared memory.
struct Coarse {
    int Lc;
    int soff[NIF_MAX_LEVELS + 1];
};

__global__ void __launch_bounds__(1024) k_encode_segments_bwd_sm(GridInfo g, Coarse cs,
                                                                 const nif_linseg* __restrict__ lin,
                                                                 const uint32_t* __restrict__ n_dev, int64_t n_max,
                                                                 const float* __restrict__ dfeats,
                                                                 float* __restrict__ dtab) {
    extern __shared__ float sacc[];
    int nsh = cs.soff[cs.Lc];
    for (int i = threadIdx.x; i < nsh; i += blockDim.x) sacc[i] = 0.f;
    __syncthreads();
    int64_t n = n_dev ? (int64_t)*n_dev : n_max;
    if (n > n_max) n = n_max;
    int per = 2 * g.P;
    for (int64_t gid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; gid < n * per;
         gid += (int64_t)gridDim.x * blockDim.x) {
        int64_t s = gid / per;
        int r = (int)(gid - s * per);
        int e = r >= g.P;
        int t = r - e * g.P;
        const float* L = reinterpret_cast<const float*>(lin + s) + 3 * e;
        float3 u = term_u(clamp01(make_float3(L[0], L[1], L[2])), t);
        const float* df = dfeats + gid * g.L * 2;
        for (int l = 0; l < g.L; l++) {
            int Nl = g.res[l];
            bool dense = (g.dense_mask >> l) & 1u;
            Cell c = cell_of(u, Nl);
            float2 gr = *reinterpret_cast<const float2*>(df + 2 * l);
            bool in_sh = l < cs.Lc;
            float* dl = in_sh ? sacc + cs.soff[l] : dtab + (int64_t)l * g.T * 2;
#pragma unroll
            for (int q = 0; q < 8; q++) {
                uint32_t row = grid_row(c.ix + (q & 1), c.iy + ((q >> 1) & 1), c.iz + ((q >> 2) & 1), Nl, dense, g.T);
                float w = ((q & 1) ? c.wx : 1.f - c.wx) * ((q & 2) ? c.wy : 1.f - c.wy) * ((q & 4) ? c.wz : 1.f - c.wz);
                if (in_sh) {
                    atomicAdd(dl + 2 * row, w * gr.x);
                    atomicAdd(dl + 2 * row + 1, w * gr.y);
                } else {
                    atomicAdd(reinterpret_cast<float2*>(dl) + row, make_float2(w * gr.x, w * gr.y));
                }
            }
        }
    }
    __syncthreads();
    for (int l = 0; l < cs.Lc; l++) {
        int cnt = cs.soff[l + 1] - cs.soff[l];
        float* dst = dtab + (int64_t)l * g.T * 2;
        for (int i = threadIdx.x; i < cnt; i += blockDim.x) {
            float v = sacc[cs.soff[l] + i];
            if (v != 0.f) atomicAdd(dst + i, v);
        }
    }
}

// Backward with a run-length register cache (the smallest dense levels,
// whose few rows every warp hits, are privatised in shared memory; a
// shared-memory float reduction costs more issue slots than a reduction in
// L2, so only levels of a few hundred rows pay off there: measured, levels of
// <= 512 rows in shared memory 1.37 ms, all five dense levels 1.59 ms, none
// 1.97 ms on the training workload). A warp owns 32/L gamma terms x
// L levels (lane = level + L * term) and walks a chunk of kRun consecutive
// segments, visiting each segment's two end points in turn: p0(s), p1(s),
// p0(s+1), ... Segments come in ray order, and where two voxels share a face
// the exit point of one is the entry point of the next (the same deformed
// point through the same inverse), so p1(s) and p0(s+1) fall in the same cell
// at every level; coarse cells also repeat over many segments. Each lane
// keeps its current cell and the running weighted sums of its 8 corners and
// reduces them into the table only when the cell changes: dense coarse levels
// into the block's shared-memory copy, the rest into global memory, where the
// two corners of an x-edge whose rows are 2m and 2m+1 (always for an even
// cell x index on a hashed level: the rows differ in bit 0 only; for an even
// base row on a dense level) share one 16-byte vector reduction. Chunks of
// points go to warps from a counter, so a warp whose chunks flushed little
// takes more of them (with a fixed stride a block's warps waited at its final
// barrier for the slowest one).
constexpr int kRun = 32;
constexpr int kFixBad = -100000;         // deterministic mode's scale word: a non-finite dL/dfeature was seen
constexpr int kFixMinS = -60, kFixMaxS = 100;

// 2^S as an FP32 value (exact: S in [kFixMinS, kFixMaxS]). A FP32 value times
// 2^S is exact wherever the rounding to an integer can matter (results of at
// least 1/2 are far above FP32's normal range limit), so the rounding gives
// what the exact product would.
__device__ __forceinline__ float fix_scale_f(int S) { return __int_as_float((S + 127) << 23); }

__device__ __forceinline__ void red_add_v2(float* addr, float a, float b) {
    asm volatile("red.global.add.v2.f32 [%0], {%1, %2};" ::"l"(addr), "f"(a), "f"(b) : "memory");
}

__device__ __forceinline__ void red_add_v4(float* addr, float a, float b, float c, float d) {
    asm volatile("red.global.add.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(addr), "f"(a), "f"(b), "f"(c), "f"(d)
                 : "memory");
}

// deterministic mode's flush: each corner sum (an FP32 value fixed by the
// chunk's points and their order) rounded to 64-bit fixed point, scale 2^S,
// and added with integer atomics, whose result does not depend on the order
__device__ __forceinline__ void flush_cell_fixed(unsigned long long* dl, int ix, int iy, int iz, int Nl, bool dense,
                                                 uint32_t T, const float2* acc, float scale) {
#pragma unroll
    for (int q = 0; q < 8; q++) {
        const uint32_t r = grid_row(ix + (q & 1), iy + ((q >> 1) & 1), iz + ((q >> 2) & 1), Nl, dense, T);
        const long long a = __float2ll_rn(acc[q].x * scale);
        const long long b = __float2ll_rn(acc[q].y * scale);
        if (a) atomicAdd(dl + 2 * r, (unsigned long long)a);
        if (b) atomicAdd(dl + 2 * r + 1, (unsigned long long)b);
    }
}

__device__ __forceinline__ void flush_cell(float* dl, bool in_sh, int ix, int iy, int iz, int Nl, bool dense,
                                           uint32_t T, const float2* acc) {
#pragma unroll
    for (int q = 0; q < 8; q += 2) {
        const uint32_t r0 = grid_row(ix, iy + ((q >> 1) & 1), iz + ((q >> 2) & 1), Nl, dense, T);
        const uint32_t r1 = grid_row(ix + 1, iy + ((q >> 1) & 1), iz + ((q >> 2) & 1), Nl, dense, T);
        if (in_sh) {
            atomicAdd(dl + 2 * r0, acc[q].x);
            atomicAdd(dl + 2 * r0 + 1, acc[q].y);
            atomicAdd(dl + 2 * r1, acc[q + 1].x);
            atomicAdd(dl + 2 * r1 + 1, acc[q + 1].y);
        } else if (r1 == (r0 ^ 1u)) {
            if (r0 & 1u) red_add_v4(dl + 2 * r1, acc[q + 1].x, acc[q + 1].y, acc[q].x, acc[q].y);
            else red_add_v4(dl + 2 * r0, acc[q].x, acc[q].y, acc[q + 1].x, acc[q + 1].y);
        } else {
            red_add_v2(dl + 2 * r0, acc[q].x, acc[q].y);
            red_add_v2(dl + 2 * r1, acc[q + 1].x, acc[q + 1].y);
        }
    }
}

// FIX (deterministic mode): the shared-memory levels and the table gradient
// are 64-bit fixed point (sfix, fix), flushed by flush_cell_fixed; the scale
// exponent comes from S_dev (k_fix_scale), and dtab is not touched.
template <bool FIX, int KS>
__global__ void __launch_bounds__(1024) k_encode_segments_bwd_rl(GridInfo g, Coarse cs,
                                                                 const nif_linseg* __restrict__ lin,
                                                                 const uint32_t* __restrict__ n_dev, int64_t n_max,
                                                                 const float* __restrict__ dfeats,
                                                                 float* __restrict__ dtab,
                                                                 const uint32_t* __restrict__ pts,
                                                                 const uint32_t* __restrict__ n_pts_dev,
                                                                 const uint32_t* __restrict__ dupf,
                                                                 uint32_t* __restrict__ next,
                                                                 unsigned long long* __restrict__ fix,
                                                                 const int* __restrict__ S_dev) {
    constexpr int ksplit = KS;
    extern __shared__ float sacc[];
    unsigned long long* sfix = reinterpret_cast<unsigned long long*>(sacc);
    float scale = 0.f;
    if (FIX) {
        const int S = *S_dev;
        if (S == kFixBad) return;                 // the conversion writes NaN gradients
        scale = fix_scale_f(S);
    }
    const int nsh = cs.soff[cs.Lc];
    for (int i = threadIdx.x; i < nsh; i += blockDim.x) {
        if (FIX) sfix[i] = 0ull;
        else sacc[i] = 0.f;
    }
    __syncthreads();
    int64_t n = n_dev ? (int64_t)*n_dev : n_max;
    if (n > n_max) n = n_max;
    const int lane = threadIdx.x & 31;
    // ksplit = 2: a task holds half of the levels (lane = level in the half +
    // L/2 * term), so a warp's fine (hashed) levels, which flush on almost
    // every point, fill all 32 lanes instead of idling beside the coarse ones
    const int LK = g.L / ksplit;                       // levels of a lane group
    const int tpw = 32 / LK;                           // gamma terms per warp
    const int groups = (g.P + tpw - 1) / tpw;
    const int lh = lane % LK;
    const int term_in_warp = lane / LK;
    // the distinct end points in order (a repeated entry point adds its
    // feature gradient to the exit point it repeats), 2 kRun per chunk
    const int64_t n_points = *n_pts_dev;
    const int64_t chunks = (n_points + 2 * kRun - 1) / (2 * kRun);
    const int64_t tasks = chunks * groups * ksplit;
    for (;;) {
        uint32_t tk = 0;
        if (lane == 0) tk = atomicAdd(next, 1u);
        const int64_t task = (int64_t)__shfl_sync(0xffffffffu, tk, 0);
        if (task >= tasks) break;
        const int64_t c = task / (groups * ksplit);
        const int rem = (int)(task - c * groups * ksplit);
        const int grp = rem / ksplit;
        const int l = (rem - grp * ksplit) * LK + lh;      // this lane's level
        const int Nl = g.res[l];
        const bool dense = (g.dense_mask >> l) & 1u;
        const bool in_sh = l < cs.Lc;
        float* dl = in_sh ? sacc + cs.soff[l] : dtab + (int64_t)l * g.T * 2;
        unsigned long long* dlf = FIX ? (in_sh ? sfix + cs.soff[l] : fix + (int64_t)l * g.T * 2) : nullptr;
        // a group with fewer terms than level groups (the last one when tpw
        // does not divide P) gives each term nr of them, each walking its own
        // part of the chunk, instead of leaving them idle
        const int a = min(g.P - grp * tpw, tpw);          // terms in this group
        const int nr = tpw / a;                           // parts per term
        const int t = grp * tpw + term_in_warp % a;       // gamma term in [0, P)
        const int sub = term_in_warp / a;                 // part of the chunk (idle when >= nr)
        const int tc = t;
        int cx = -1, cy = 0, cz = 0;                      // current cell (cx < 0: none)
        float2 cacc[8];
#pragma unroll
        for (int q = 0; q < 8; q++) cacc[q] = make_float2(0.f, 0.f);
        const int64_t k0 = c * 2 * kRun;
        const int span = (int)(k0 + 2 * kRun < n_points ? 2 * kRun : n_points - k0);
        const int part = (span + nr - 1) / nr;
        const int kb = sub < nr ? sub * part : span;      // this part's points: k0 + [kb, ke)
        const int ke = min(kb + part, span);
        const int base = term_in_warp * LK;               // first lane of this term's level group
        for (int i = 0; i < part; i++) {                  // warp-uniform trip count (shuffles below)
            const bool active = kb + i < ke;
            {
                const uint32_t pt = pts[k0 + (active ? kb + i : 0)];
                const int64_t s = pt >> 1;
                const int e = (int)(pt & 1);
                // the term's u is the same for all L levels: lanes base..base+2
                // evaluate one coordinate each and the group shares them
                const float* Lp = reinterpret_cast<const float*>(lin + s) + 3 * e;
                const int cc = lh < 3 ? lh : 0;
                const float pc = fminf(fmaxf(Lp[cc], 0.f), 1.f);
                float uc;
                if (tc == 0) {
                    uc = pc;
                } else {
                    const float f = (float)(1 << ((tc - 1) >> 1));
                    float sn, cn;
                    sincosf(f * pc, &sn, &cn);
                    uc = (((tc - 1) & 1) ? cn + 1.0f : sn + 1.0f) * 0.5f;
                }
                float3 u;
                u.x = __shfl_sync(0xffffffffu, uc, base);
                u.y = __shfl_sync(0xffffffffu, uc, base + 1);
                u.z = __shfl_sync(0xffffffffu, uc, base + 2);
                if (!active) continue;
                Cell cl = cell_of(u, Nl);
                float2 gr = *reinterpret_cast<const float2*>(dfeats + ((s * 2 * g.P + e * g.P + t) * g.L + l) * 2);
                if (e == 1 && s + 1 < n_max && dupf[s + 1] == 1) {
                    const float2 g2 = *reinterpret_cast<const float2*>(dfeats + (((s + 1) * 2 * g.P + t) * g.L + l) * 2);
                    gr.x += g2.x;
                    gr.y += g2.y;
                }
                if (cl.ix != cx || cl.iy != cy || cl.iz != cz) {
                    if (cx >= 0) {
                        if (FIX) flush_cell_fixed(dlf, cx, cy, cz, Nl, dense, g.T, cacc, scale);
                        else flush_cell(dl, in_sh, cx, cy, cz, Nl, dense, g.T, cacc);
                    }
                    cx = cl.ix;
                    cy = cl.iy;
                    cz = cl.iz;
#pragma unroll
                    for (int q = 0; q < 8; q++) cacc[q] = make_float2(0.f, 0.f);
                }
                // corner weights (x fastest, the same products as one at a
                // time) and both features of a corner in one packed FP32 FMA
                const float2 wx = make_float2(1.f - cl.wx, cl.wx);
                const float wy0 = 1.f - cl.wy, wy1 = cl.wy, wz0 = 1.f - cl.wz, wz1 = cl.wz;
                const float2 wxy0 = __fmul2_rn(wx, make_float2(wy0, wy0));
                const float2 wxy1 = __fmul2_rn(wx, make_float2(wy1, wy1));
                const float2 wq[4] = {__fmul2_rn(wxy0, make_float2(wz0, wz0)), __fmul2_rn(wxy1, make_float2(wz0, wz0)),
                                      __fmul2_rn(wxy0, make_float2(wz1, wz1)), __fmul2_rn(wxy1, make_float2(wz1, wz1))};
#pragma unroll
                for (int q = 0; q < 8; q++) {
                    const float w = (q & 1) ? wq[q >> 1].y : wq[q >> 1].x;
                    cacc[q] = __ffma2_rn(make_float2(w, w), gr, cacc[q]);
                }
            }
        }
        if (cx >= 0) {
            if (FIX) flush_cell_fixed(dlf, cx, cy, cz, Nl, dense, g.T, cacc, scale);
            else flush_cell(dl, in_sh, cx, cy, cz, Nl, dense, g.T, cacc);
        }
    }
    __syncthreads();
    for (int lv = 0; lv < cs.Lc; lv++) {
        int cnt = cs.soff[lv + 1] - cs.soff[lv];
        for (int i = threadIdx.x; i < cnt; i += blockDim.x) {
            if (FIX) {
                const unsigned long long v = sfix[cs.soff[lv] + i];
                if (v) atomicAdd(fix + (int64_t)lv * g.T * 2 + i, v);
            } else {
                float v = sacc[cs.soff[lv] + i];
                if (v != 0.f) atomicAdd(dtab + (int64_t)lv * g.T * 2 + i, v);
            }
        }
    }
}

// Input gradient of the segment encoding with the tables held fixed:
// dp[s][e][3] += d(sum dfeats * psi)/d p_e of segment s (zero where clamped).
__global__ void __launch_bounds__(256) k_encode_segments_dp(GridInfo g, const float* __restrict__ tab,
                                                            const nif_linseg* __restrict__ lin,
                                                            const uint32_t* __restrict__ n_dev, int64_t n_max,
                                                            const float* __restrict__ dfeats,
                                                            float* __restrict__ dp) {
    int64_t n = n_dev ? (int64_t)*n_dev : n_max;
    if (n > n_max) n = n_max;
    int per = 2 * g.P;
    for (int64_t gid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; gid < n * per;
         gid += (int64_t)gridDim.x * blockDim.x) {
        int64_t s = gid / per;
        int r = (int)(gid - s * per);
        int e = r >= g.P;
        int t = r - e * g.P;
        const float* L = reinterpret_cast<const float*>(lin + s) + 3 * e;
        float3 raw = make_float3(L[0], L[1], L[2]);
        float3 p = clamp01(raw);
        float3 u = term_u(p, t);
        float3 du = make_float3(0.f, 0.f, 0.f);
        const float* df = dfeats + gid * g.L * 2;
        for (int l = 0; l < g.L; l++) {
            int Nl = g.res[l];
            bool dense = (g.dense_mask >> l) & 1u;
            Cell c = cell_of(u, Nl);
            float2 gr = *reinterpret_cast<const float2*>(df + 2 * l);
            const float* tl = tab + (int64_t)l * g.T * 2;
            float3 d = make_float3(0.f, 0.f, 0.f);
#pragma unroll
            for (int q = 0; q < 8; q++) {
                uint32_t row = grid_row(c.ix + (q & 1), c.iy + ((q >> 1) & 1), c.iz + ((q >> 2) & 1), Nl, dense, g.T);
                float fx = (q & 1) ? c.wx : 1.f - c.wx;
                float fy = (q & 2) ? c.wy : 1.f - c.wy;
                float fz = (q & 4) ? c.wz : 1.f - c.wz;
                float2 v = __ldg(reinterpret_cast<const float2*>(tl) + row);
                float val = v.x * gr.x + v.y * gr.y;
                d.x += ((q & 1) ? 1.f : -1.f) * fy * fz * val;
                d.y += ((q & 2) ? 1.f : -1.f) * fx * fz * val;
                d.z += ((q & 4) ? 1.f : -1.f) * fx * fy * val;
            }
            float fn = (float)Nl;
            du.x += fn * d.x;
            du.y += fn * d.y;
            du.z += fn * d.z;
        }
        float3 j = term_dudp(p, t);
        if (raw.x < 0.f || raw.x > 1.f) j.x = 0.f;
        if (raw.y < 0.f || raw.y > 1.f) j.y = 0.f;
        if (raw.z < 0.f || raw.z > 1.f) j.z = 0.f;
        float* o = dp + s * 6 + e * 3;
        atomicAdd(o, du.x * j.x);
        atomicAdd(o + 1, du.y * j.y);
        atomicAdd(o + 2, du.z * j.z);
    }
}

template <typename TT, typename OT>
void launch_points(nif_handle* h, const TT* tab, const float* pts, int64_t n, void* feats, int32_t* rows,
                   cudaStream_t s) {
    k_encode_points<TT, OT><<<nif_blocks(n * h->P, 256), 256, 0, s>>>(h->grid, tab, pts, n, (OT*)feats, rows);
}

// The list of distinct end points of segments [0, n) (flags in *dupf, count in
// *n_pts on the device) in the handle's scratch.
nif_status distinct_points(nif_handle* h, const nif_linseg* lin, const uint32_t* n_dev, int64_t n_max,
                           const uint32_t** pts_out, const uint32_t** n_pts_out, const uint32_t** dupf_out,
                           cudaStream_t s) {
    nif_status st;
    h->enc_points = nif_handle::PointList{};             // its buffers are rewritten here
    if ((st = nif_grow(h, h->b_dup, sizeof(uint32_t) * (2 * (size_t)n_max + 1))) != NIF_OK) return st;
    if ((st = nif_grow(h, h->b_pts, sizeof(uint32_t) * 2 * (size_t)n_max)) != NIF_OK) return st;
    const int nb = (int)nif_blocks(n_max, 1024);
    if ((st = nif_grow(h, h->b_scan, sizeof(uint32_t) * ((size_t)nb + 1))) != NIF_OK) return st;
    uint32_t* u = (uint32_t*)h->b_dup.p;
    uint32_t* off = u + n_max;
    uint32_t* pts = (uint32_t*)h->b_pts.p;
    unsigned gs = std::min<unsigned>(nif_blocks(n_max, 256), (unsigned)h->num_sms * 16);
    k_dup_flags<<<gs, 256, 0, s>>>(lin, n_dev, n_max, u);
    NIF_CK_LAUNCH(h);
    if ((st = nif_scan_run_with(h, u, off, (int)n_max, (uint32_t*)h->b_scan.p, s)) != NIF_OK) return st;
    k_point_list<<<gs, 256, 0, s>>>(u, off, n_max, pts);
    NIF_CK_LAUNCH(h);
    *pts_out = pts;
    *n_pts_out = off + n_max;
    *dupf_out = u;
    return NIF_OK;
}

// The distinct points in rest-space order: a counting sort by the Morton
// code of each point's cell in a 2^b x 2^b x 2^b grid over the cube
// (b = NIF_KNOB_ORDER_BITS, default 7: a finer grid keeps the backward's
// cell cache on one cell longer at the middle levels). A warp of the encoder then takes 32
// points of one small region, whose corner rows at the coarse levels (and
// the low bands of gamma) coincide, so their loads merge into far fewer L1
// wavefronts than points taken along rays; the gather is bound by L1
// wavefronts. The order within a cell is arbitrary and does not matter:
// every point's features go to its own rows.
__device__ __forceinline__ uint32_t spread3(uint32_t v) {     // bits 0..9 of v to bits 0, 3, 6, ...
    v &= 0x3FFu;
    v = (v | (v << 16)) & 0x030000FFu;
    v = (v | (v << 8)) & 0x0300F00Fu;
    v = (v | (v << 4)) & 0x030C30C3u;
    v = (v | (v << 2)) & 0x09249249u;
    return v;
}

__global__ void __launch_bounds__(256) k_point_keys(const nif_linseg* __restrict__ lin, const uint32_t* __restrict__ pts,
                                                    const uint32_t* __restrict__ n_pts_dev, int bits,
                                                    uint32_t* __restrict__ keys, uint32_t* __restrict__ hist) {
    const int64_t n = *n_pts_dev;
    const float cells = (float)(1 << bits);
    const uint32_t top = (1u << bits) - 1u;
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t pt = pts[k];
        const float* L = reinterpret_cast<const float*>(lin + (pt >> 1)) + 3 * (pt & 1u);
        const float3 p = clamp01(make_float3(L[0], L[1], L[2]));
        const uint32_t ix = min((uint32_t)(p.x * cells), top);
        const uint32_t iy = min((uint32_t)(p.y * cells), top);
        const uint32_t iz = min((uint32_t)(p.z * cells), top);
        const uint32_t key = spread3(ix) | (spread3(iy) << 1) | (spread3(iz) << 2);
        keys[k] = key;
        atomicAdd(hist + key, 1u);
    }
}

__global__ void __launch_bounds__(256) k_point_scatter(const uint32_t* __restrict__ pts,
                                                       const uint32_t* __restrict__ n_pts_dev,
                                                       const uint32_t* __restrict__ keys,
                                                       const uint32_t* __restrict__ off, uint32_t* __restrict__ fill,
                                                       uint32_t* __restrict__ sorted) {
    const int64_t n = *n_pts_dev;
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t key = keys[k];
        const uint32_t at = off[key] + atomicAdd(fill + key, 1u);
        if (NIF_IN(at, n)) sorted[at] = pts[k];
    }
}

// Deterministic mode: the scatter above leaves a cell's points in the order
// the atomics gave them; each cell's run is put in ascending point order (one
// thread a cell, insertion sort: cells hold a few points each), so the order,
// and with it every float sum the backward forms along it, is fixed.
__global__ void __launch_bounds__(256) k_point_cell_sort(const uint32_t* __restrict__ off, int64_t cells,
                                                         uint32_t* __restrict__ sorted) {
    for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < cells; c += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t a = off[c], b = off[c + 1];
        for (uint32_t i = a + 1; i < b; i++) {
            const uint32_t v = sorted[i];
            uint32_t j = i;
            while (j > a && sorted[j - 1] > v) {
                sorted[j] = sorted[j - 1];
                j--;
            }
            sorted[j] = v;
        }
    }
}

// sorted (out): the *n_pts_dev points of pts in rest-space order
nif_status spatial_order(nif_handle* h, const nif_linseg* lin, const uint32_t* pts, const uint32_t* n_pts_dev,
                         int64_t n_max, const uint32_t** sorted_out, cudaStream_t s) {
    const size_t np = 2 * (size_t)n_max;
    const int bits = h->tune.order_bits;
    const size_t cells = (size_t)1 << (3 * bits);
    const size_t nbs = cells / 1024 + 2;
    nif_status st = nif_grow(h, h->b_sort, sizeof(uint32_t) * (2 * np + 2 * cells + 1 + nbs));
    if (st != NIF_OK) return st;
    uint32_t* keys = (uint32_t*)h->b_sort.p;
    uint32_t* sorted = keys + np;
    uint32_t* hist = sorted + np;
    uint32_t* off = hist + cells;
    uint32_t* bsum = off + cells + 1;
    const unsigned g = std::min<unsigned>(nif_blocks((int64_t)np, 256), (unsigned)h->num_sms * 8);
    NIF_CK(h, cudaMemsetAsync(hist, 0, sizeof(uint32_t) * cells, s));
    k_point_keys<<<g, 256, 0, s>>>(lin, pts, n_pts_dev, bits, keys, hist);
    NIF_CK_LAUNCH(h);
    if ((st = nif_scan_run_with(h, hist, off, (int)cells, bsum, s)) != NIF_OK) return st;
    NIF_CK(h, cudaMemsetAsync(hist, 0, sizeof(uint32_t) * cells, s));
    k_point_scatter<<<g, 256, 0, s>>>(pts, n_pts_dev, keys, off, hist, sorted);
    NIF_CK_LAUNCH(h);
    if (h->det) {
        k_point_cell_sort<<<(unsigned)std::min<int64_t>(nif_blocks((int64_t)cells, 256), (int64_t)h->num_sms * 8), 256,
                            0, s>>>(off, (int64_t)cells, sorted);
        NIF_CK_LAUNCH(h);
    }
    *sorted_out = sorted;
    return NIF_OK;
}

// The distinct end points of lin's segments, in rest-space order when the
// tables (of table_bytes per entry) exceed 4 MiB: tables of a few MB stay in
// L1 and L2 in any order (measured: the sort costs the 1 MiB-table query 5 %);
// larger ones gain from it (the 32 MiB tables of the 64-instance batch:
// encoder 1.35x faster). Recorded in h->enc_points.
static nif_status point_list(nif_handle* h, const nif_linseg* lin, const uint32_t* n_dev, int64_t n_max,
                             size_t table_bytes, cudaStream_t s) {
    const uint32_t *pts = nullptr, *n_pts = nullptr, *dupf = nullptr;
    nif_status st = distinct_points(h, lin, n_dev, n_max, &pts, &n_pts, &dupf, s);
    if (st != NIF_OK) return st;
    const bool sorted = (size_t)h->T * h->L * h->Fd * table_bytes > ((size_t)4 << 20);
    if (sorted && (st = spatial_order(h, lin, pts, n_pts, n_max, &pts, s)) != NIF_OK) return st;
    h->enc_points = nif_handle::PointList{lin, n_dev, n_max, pts, n_pts, dupf, sorted};
    return NIF_OK;
}

template <typename TT, typename OT>
nif_status launch_segments(nif_handle* h, const TT* tab, const nif_linseg* lin, const uint32_t* n_dev, int64_t n_max,
                           void* feats, cudaStream_t s, bool reuse_points, bool dedup) {
    // block size and resident blocks per SM are tuning knobs of the handle
    int thr = h->tune.enc_threads;
    unsigned g = nif_blocks(n_max * 2 * h->P, thr);
    unsigned cap = (unsigned)h->num_sms * (unsigned)h->tune.enc_blocks_per_sm;
    if (g > cap) g = cap;
    if (h->L <= 16 && !dedup) {
        // every (segment, end point): no point list to prepare, so a chunk
        // whose device count is zero costs one early-exiting launch
        if (h->L <= 8)
            k_encode_segments_v<TT, OT, 8><<<g, thr, 0, s>>>(h->grid, tab, lin, n_dev, n_max, (OT*)feats, nullptr,
                                                            nullptr, nullptr);
        else
            k_encode_segments_v<TT, OT, 16><<<g, thr, 0, s>>>(h->grid, tab, lin, n_dev, n_max, (OT*)feats, nullptr,
                                                             nullptr, nullptr);
    } else if (h->L <= 16) {
        // distinct end points only (device-side list, see k_dup_flags)
        const nif_handle::PointList& pl = h->enc_points;
        const bool sorted = (size_t)h->T * h->L * h->Fd * sizeof(TT) > ((size_t)4 << 20);
        if (!(reuse_points && pl.pts && pl.lin == lin && pl.n_dev == n_dev && pl.n_max == n_max &&
              pl.sorted == sorted)) {
            nif_status st = point_list(h, lin, n_dev, n_max, sizeof(TT), s);
            if (st != NIF_OK) return st;
        }
        const uint32_t *pts = pl.pts, *n_pts = pl.n_pts, *dupf = pl.dupf;
        if (h->L <= 8)
            k_encode_segments_v<TT, OT, 8><<<g, thr, 0, s>>>(h->grid, tab, lin, n_dev, n_max, (OT*)feats, pts,
                                                            n_pts, dupf);
        else
            k_encode_segments_v<TT, OT, 16><<<g, thr, 0, s>>>(h->grid, tab, lin, n_dev, n_max, (OT*)feats, pts,
                                                             n_pts, dupf);
    } else
        k_encode_segments<TT, OT><<<g, thr, 0, s>>>(h->grid, tab, lin, n_dev, n_max, (OT*)feats);
    return NIF_OK;
}

// ---------------------------------------------------------------------------
// The concatenation reading of Eq. 1: psi(p) = [gamma(p), phi(p)]. A segment's
// row is [psi(p0) | psi(p1) | zeros] of in_dim columns, W = 3P + L*F_d per
// end point: gamma's raw values ordered [term][coordinate] (x, then
// sin(2^k x), cos(2^k x) for k < F) and the grid features at u = p (p
// clamped to [0,1]^3), ordered [level][feature].
// ---------------------------------------------------------------------------
template <typename OT>
__device__ __forceinline__ OT to_out(float v);
template <>
__device__ __forceinline__ float to_out<float>(float v) { return v; }
template <>
__device__ __forceinline__ __nv_bfloat16 to_out<__nv_bfloat16>(float v) { return __float2bfloat16_rn(v); }
template <>
__device__ __forceinline__ __half to_out<__half>(float v) { return __float2half_rn(v); }

// one thread per (segment, end point)
template <typename TT, typename OT>
__global__ void __launch_bounds__(256) k_encode_cat(GridInfo g, const TT* __restrict__ tab,
                                                    const nif_linseg* __restrict__ lin,
                                                    const uint32_t* __restrict__ n_dev, int64_t n_max, int in_dim,
                                                    OT* __restrict__ out) {
    int64_t n = n_dev ? (int64_t)*n_dev : n_max;
    if (n > n_max) n = n_max;
    const int W = 3 * g.P + g.L * 2;
    for (int64_t gid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; gid < 2 * n;
         gid += (int64_t)gridDim.x * blockDim.x) {
        const int64_t s = gid >> 1;
        const int e = (int)(gid & 1);
        const float* L = reinterpret_cast<const float*>(lin + s) + 3 * e;
        const float3 p = clamp01(make_float3(L[0], L[1], L[2]));
        OT* row = out + s * in_dim + e * W;
        row[0] = to_out<OT>(p.x);
        row[1] = to_out<OT>(p.y);
        row[2] = to_out<OT>(p.z);
        for (int k = 0; k < g.F; k++) {
            const float f = (float)(1 << k);
            float sx, cx, sy, cy, sz, cz;
            sincosf(f * p.x, &sx, &cx);
            sincosf(f * p.y, &sy, &cy);
            sincosf(f * p.z, &sz, &cz);
            OT* r = row + 3 + 6 * k;
            r[0] = to_out<OT>(sx); r[1] = to_out<OT>(sy); r[2] = to_out<OT>(sz);
            r[3] = to_out<OT>(cx); r[4] = to_out<OT>(cy); r[5] = to_out<OT>(cz);
        }
        OT* fr = row + 3 * g.P;
        for (int l = 0; l < g.L; l++) {
            const int Nl = g.res[l];
            const bool dense = (g.dense_mask >> l) & 1u;
            const Cell c = cell_of(p, Nl);
            const TT* tl = tab + (int64_t)l * g.T * 2;
            float2 acc = make_float2(0.f, 0.f);
#pragma unroll
            for (int q = 0; q < 8; q++) {
                const uint32_t rw = grid_row(c.ix + (q & 1), c.iy + ((q >> 1) & 1), c.iz + ((q >> 2) & 1), Nl, dense, g.T);
                const float w = ((q & 1) ? c.wx : 1.f - c.wx) * ((q & 2) ? c.wy : 1.f - c.wy) *
                                ((q & 4) ? c.wz : 1.f - c.wz);
                const float2 v = load_row<TT>(tl, rw);
                acc.x += w * v.x;
                acc.y += w * v.y;
            }
            fr[2 * l] = to_out<OT>(acc.x);
            fr[2 * l + 1] = to_out<OT>(acc.y);
        }
        if (e == 1)
            for (int j = 2 * W; j < in_dim; j++) out[s * in_dim + j] = to_out<OT>(0.f);
    }
}

// table gradient of the phi part: one thread per (segment, end point, level)
__global__ void __launch_bounds__(256) k_encode_cat_bwd(GridInfo g, const nif_linseg* __restrict__ lin,
                                                        const uint32_t* __restrict__ n_dev, int64_t n_max, int in_dim,
                                                        const float* __restrict__ dfeats, float* __restrict__ dtab) {
    int64_t n = n_dev ? (int64_t)*n_dev : n_max;
    if (n > n_max) n = n_max;
    const int W = 3 * g.P + g.L * 2;
    const int per = 2 * g.L;
    for (int64_t gid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; gid < n * per;
         gid += (int64_t)gridDim.x * blockDim.x) {
        const int64_t s = gid / per;
        const int r = (int)(gid - s * per);
        const int e = r / g.L, l = r - e * g.L;
        const float* L = reinterpret_cast<const float*>(lin + s) + 3 * e;
        const float3 p = clamp01(make_float3(L[0], L[1], L[2]));
        const float* df = dfeats + s * in_dim + e * W + 3 * g.P + 2 * l;
        const float gx = df[0], gy = df[1];
        const int Nl = g.res[l];
        const bool dense = (g.dense_mask >> l) & 1u;
        const Cell c = cell_of(p, Nl);
        float2* dl = reinterpret_cast<float2*>(dtab + (int64_t)l * g.T * 2);
#pragma unroll
        for (int q = 0; q < 8; q++) {
            const uint32_t rw = grid_row(c.ix + (q & 1), c.iy + ((q >> 1) & 1), c.iz + ((q >> 2) & 1), Nl, dense, g.T);
            const float w = ((q & 1) ? c.wx : 1.f - c.wx) * ((q & 2) ? c.wy : 1.f - c.wy) *
                            ((q & 4) ? c.wz : 1.f - c.wz);
            atomicAdd(dl + rw, make_float2(w * gx, w * gy));
        }
    }
}

// input gradient with the tables fixed: dp[s][e][3] = d(sum dfeats * psi)/d p_e
// (gamma's derivative plus the grid's), zero where p was clamped
__global__ void __launch_bounds__(256) k_encode_cat_dp(GridInfo g, const float* __restrict__ tab,
                                                       const nif_linseg* __restrict__ lin,
                                                       const uint32_t* __restrict__ n_dev, int64_t n_max, int in_dim,
                                                       const float* __restrict__ dfeats, float* __restrict__ dp) {
    int64_t n = n_dev ? (int64_t)*n_dev : n_max;
    if (n > n_max) n = n_max;
    const int W = 3 * g.P + g.L * 2;
    for (int64_t gid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; gid < 2 * n;
         gid += (int64_t)gridDim.x * blockDim.x) {
        const int64_t s = gid >> 1;
        const int e = (int)(gid & 1);
        const float* L = reinterpret_cast<const float*>(lin + s) + 3 * e;
        const float3 raw = make_float3(L[0], L[1], L[2]);
        const float3 p = clamp01(raw);
        const float* df = dfeats + s * in_dim + e * W;
        float3 d = make_float3(df[0], df[1], df[2]);
        for (int k = 0; k < g.F; k++) {
            const float f = (float)(1 << k);
            float sx, cx, sy, cy, sz, cz;
            sincosf(f * p.x, &sx, &cx);
            sincosf(f * p.y, &sy, &cy);
            sincosf(f * p.z, &sz, &cz);
            const float* r = df + 3 + 6 * k;
            d.x += f * (r[0] * cx - r[3] * sx);
            d.y += f * (r[1] * cy - r[4] * sy);
            d.z += f * (r[2] * cz - r[5] * sz);
        }
        const float* fr = df + 3 * g.P;
        for (int l = 0; l < g.L; l++) {
            const int Nl = g.res[l];
            const bool dense = (g.dense_mask >> l) & 1u;
            const Cell c = cell_of(p, Nl);
            const float gx = fr[2 * l], gy = fr[2 * l + 1];
            const float* tl = tab + (int64_t)l * g.T * 2;
            float3 dl = make_float3(0.f, 0.f, 0.f);
#pragma unroll
            for (int q = 0; q < 8; q++) {
                const uint32_t rw = grid_row(c.ix + (q & 1), c.iy + ((q >> 1) & 1), c.iz + ((q >> 2) & 1), Nl, dense, g.T);
                const float fx = (q & 1) ? c.wx : 1.f - c.wx;
                const float fy = (q & 2) ? c.wy : 1.f - c.wy;
                const float fz = (q & 4) ? c.wz : 1.f - c.wz;
                const float2 v = __ldg(reinterpret_cast<const float2*>(tl) + rw);
                const float val = v.x * gx + v.y * gy;
                dl.x += ((q & 1) ? 1.f : -1.f) * fy * fz * val;
                dl.y += ((q & 2) ? 1.f : -1.f) * fx * fz * val;
                dl.z += ((q & 4) ? 1.f : -1.f) * fx * fy * val;
            }
            const float fn = (float)Nl;
            d.x += fn * dl.x;
            d.y += fn * dl.y;
            d.z += fn * dl.z;
        }
        float* o = dp + s * 6 + e * 3;
        o[0] = (raw.x < 0.f || raw.x > 1.f) ? 0.f : d.x;
        o[1] = (raw.y < 0.f || raw.y > 1.f) ? 0.f : d.y;
        o[2] = (raw.z < 0.f || raw.z > 1.f) ? 0.f : d.z;
    }
}


// ---------------------------------------------------------------------------
// Deterministic table gradient (NIF_KNOB_DETERMINISTIC). Float reductions in
// L2 add in whatever order the warps reach them, so two runs of one step can
// differ in the last bits of the sums. Here each contribution w * dL/dfeature
// (the same FP32 product as above) is scaled by 2^S, rounded once to a 64-bit
// integer and added with integer atomics; integer addition is associative,
// so the sum and the FP32 value it converts to do not depend on the order.
// S comes from M = max |dL/dfeature| of the call: a table entry of level l
// takes at most one weighted term per (segment, end point, gamma term), with
// trilinear weights summing to at most 1 over the cell's corners, so every
// sum is bounded by 2 n P M; S is the largest integer with 2 n P M 2^S <
// 2^61, which leaves the rounding (at most 1/2 per contribution) far from
// overflow. Each contribution's rounding error is at most 2^-(S+1).
// ---------------------------------------------------------------------------

// *bits = max over the first min(*n_dev, n_max) * per floats of x of the bit
// pattern of |x| (the order of non-negative floats; NaN compares above inf)
__global__ void __launch_bounds__(256) k_absmax_bits(const float* __restrict__ x, const uint32_t* __restrict__ n_dev,
                                                     int64_t n_max, int64_t per, uint32_t* __restrict__ bits) {
    int64_t n = n_dev ? (int64_t)*n_dev : n_max;
    if (n > n_max) n = n_max;
    const int64_t cnt = n * per;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t i0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    uint32_t m = 0;
    if ((reinterpret_cast<uintptr_t>(x) & 15u) == 0 && cnt % 4 == 0) {
        const float4* x4 = reinterpret_cast<const float4*>(x);
        for (int64_t i = i0; i < cnt / 4; i += stride) {
            const float4 v = x4[i];
            m = max(m, max(max(__float_as_uint(v.x) & 0x7fffffffu, __float_as_uint(v.y) & 0x7fffffffu),
                           max(__float_as_uint(v.z) & 0x7fffffffu, __float_as_uint(v.w) & 0x7fffffffu)));
        }
    } else {
        for (int64_t i = i0; i < cnt; i += stride) m = max(m, __float_as_uint(x[i]) & 0x7fffffffu);
    }
    m = __reduce_max_sync(0xffffffffu, m);
    if ((threadIdx.x & 31) == 0 && m) atomicMax(bits, m);
}

// the scale exponent S of the call (see above), or kFixBad
__global__ void k_fix_scale(const uint32_t* __restrict__ bits, const uint32_t* __restrict__ n_dev, int64_t n_max,
                            int P, int* __restrict__ S_out) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    int64_t n = n_dev ? (int64_t)*n_dev : n_max;
    if (n > n_max) n = n_max;
    const uint32_t b = *bits;
    if (b >= 0x7f800000u) { *S_out = kFixBad; return; }
    const double B = 2.0 * (double)n * (double)P * (double)__uint_as_float(b);
    if (B == 0.0) { *S_out = 0; return; }      // every contribution is zero
    int E = 0;
    frexp(B, &E);                              // B = m 2^E, 1/2 <= m < 1, so B 2^(61-E) < 2^61
    // a smaller S only coarsens the rounding; an S below the lowest would mean
    // gradients near FP32's range limit, treated as non-finite
    *S_out = 61 - E < kFixMinS ? kFixBad : min(61 - E, kFixMaxS);
}

// One thread per (segment, end point, gamma term), as k_encode_segments_bwd_sm:
// the dense coarse levels of cs go to the block's shared-memory copy, the rest
// to fix, both as 64-bit fixed point.
__global__ void __launch_bounds__(1024) k_encode_bwd_fixed(GridInfo g, Coarse cs, const nif_linseg* __restrict__ lin,
                                                           const uint32_t* __restrict__ n_dev, int64_t n_max,
                                                           const float* __restrict__ dfeats,
                                                           unsigned long long* __restrict__ fix,
                                                           const int* __restrict__ S_dev) {
    extern __shared__ unsigned long long sfix[];
    const int S = *S_dev;
    if (S == kFixBad) return;                  // the conversion writes NaN gradients
    const float scale = fix_scale_f(S);
    const int nsh = cs.soff[cs.Lc];
    for (int i = threadIdx.x; i < nsh; i += blockDim.x) sfix[i] = 0ull;
    __syncthreads();
    int64_t n = n_dev ? (int64_t)*n_dev : n_max;
    if (n > n_max) n = n_max;
    const int per = 2 * g.P;
    for (int64_t gid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; gid < n * per;
         gid += (int64_t)gridDim.x * blockDim.x) {
        const int64_t s = gid / per;
        const int r = (int)(gid - s * per);
        const int e = r >= g.P;
        const int t = r - e * g.P;
        const float* L = reinterpret_cast<const float*>(lin + s) + 3 * e;
        const float3 u = term_u(clamp01(make_float3(L[0], L[1], L[2])), t);
        const float* df = dfeats + gid * g.L * 2;
        for (int l = 0; l < g.L; l++) {
            const int Nl = g.res[l];
            const bool dense = (g.dense_mask >> l) & 1u;
            const Cell c = cell_of(u, Nl);
            const float2 gr = *reinterpret_cast<const float2*>(df + 2 * l);
            if (gr.x == 0.f && gr.y == 0.f) continue;
            unsigned long long* dl = l < cs.Lc ? sfix + cs.soff[l] : fix + (int64_t)l * g.T * 2;
#pragma unroll
            for (int q = 0; q < 8; q++) {
                const uint32_t row = grid_row(c.ix + (q & 1), c.iy + ((q >> 1) & 1), c.iz + ((q >> 2) & 1), Nl, dense, g.T);
                const float w = ((q & 1) ? c.wx : 1.f - c.wx) * ((q & 2) ? c.wy : 1.f - c.wy) * ((q & 4) ? c.wz : 1.f - c.wz);
                const long long a = __float2ll_rn((w * gr.x) * scale);
                const long long b = __float2ll_rn((w * gr.y) * scale);
                if (a) atomicAdd(dl + 2 * row, (unsigned long long)a);
                if (b) atomicAdd(dl + 2 * row + 1, (unsigned long long)b);
            }
        }
    }
    __syncthreads();
    for (int l = 0; l < cs.Lc; l++) {
        const int cnt = cs.soff[l + 1] - cs.soff[l];
        unsigned long long* dst = fix + (int64_t)l * g.T * 2;
        for (int i = threadIdx.x; i < cnt; i += blockDim.x) {
            const unsigned long long v = sfix[cs.soff[l] + i];
            if (v) atomicAdd(dst + i, v);
        }
    }
}

// dtab[i] += fix[i] 2^-S, and fix[i] = 0 for the next call; NaN everywhere
// when the call saw a non-finite dL/dfeature
__global__ void __launch_bounds__(256) k_fix_to_float(unsigned long long* __restrict__ fix, int64_t cnt,
                                                      const int* __restrict__ S_dev, float* __restrict__ dtab) {
    const int S = *S_dev;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < cnt; i += (int64_t)gridDim.x * blockDim.x) {
        const unsigned long long v = fix[i];
        if (S == kFixBad) {
            dtab[i] = __int_as_float(0x7fffffff);
            if (v) fix[i] = 0ull;
        } else if (v) {
            dtab[i] += (float)ldexp((double)(long long)v, -S);
            fix[i] = 0ull;
        }
    }
}

}  // namespace

nif_status nif_encode_points_prepare(nif_handle* h, const nif_linseg* lin, const uint32_t* n_dev, int64_t n_max,
                                     int table_dtype, cudaStream_t s) {
    if (n_max <= 0 || h->concat || h->L > 16) return NIF_OK;
    return point_list(h, lin, n_dev, n_max, table_dtype == NIF_FP16 ? 2 : 4, s);
}


nif_status nif_encode_points_run(nif_handle* h, const float* pts, int64_t n, void* feats, int out_dtype,
                                 int32_t* rows, cudaStream_t s) {
    NifProf prof_(h, "encode_points", s);
    if (n <= 0) return NIF_OK;
    if (h->concat) return nif_fail(h, NIF_ERR_ARG, "point encoding is the composed reading; this handle concatenates");
    const float* tab = h->d_params + h->off_tables;
    if (out_dtype == NIF_FP32) launch_points<float, float>(h, tab, pts, n, feats, rows, s);
    else if (out_dtype == NIF_BF16) launch_points<float, __nv_bfloat16>(h, tab, pts, n, feats, rows, s);
    else if (out_dtype == NIF_FP16) launch_points<float, __half>(h, tab, pts, n, feats, rows, s);
    else return nif_fail(h, NIF_ERR_ARG, "out_dtype");
    NIF_CK_LAUNCH(h);
    return NIF_OK;
}

// forward of the concatenation reading: FP32 master tables or their FP16 copy, FP32/BF16/FP16 rows
static nif_status launch_cat(nif_handle* h, const nif_linseg* lin, const uint32_t* n_dev, int64_t n_max, void* feats,
                             int out_dtype, int table_dtype, cudaStream_t s) {
    const unsigned g = (unsigned)std::min<int64_t>(nif_blocks(2 * n_max, 256), (int64_t)h->num_sms * 16);
    if (table_dtype != NIF_FP32 && table_dtype != NIF_FP16) return nif_fail(h, NIF_ERR_ARG, "table_dtype");
    if (out_dtype != NIF_FP32 && out_dtype != NIF_BF16 && out_dtype != NIF_FP16) return nif_fail(h, NIF_ERR_ARG, "out_dtype");
    if (table_dtype == NIF_FP16) {
        nif_status st = nif_refresh_lowp(h, s);
        if (st != NIF_OK) return st;
        const __half* tab = h->d_tables_h;
        if (out_dtype == NIF_FP32) k_encode_cat<__half, float><<<g, 256, 0, s>>>(h->grid, tab, lin, n_dev, n_max, h->in_dim, (float*)feats);
        else if (out_dtype == NIF_BF16) k_encode_cat<__half, __nv_bfloat16><<<g, 256, 0, s>>>(h->grid, tab, lin, n_dev, n_max, h->in_dim, (__nv_bfloat16*)feats);
        else k_encode_cat<__half, __half><<<g, 256, 0, s>>>(h->grid, tab, lin, n_dev, n_max, h->in_dim, (__half*)feats);
    } else {
        const float* tab = h->d_params + h->off_tables;
        if (out_dtype == NIF_FP32) k_encode_cat<float, float><<<g, 256, 0, s>>>(h->grid, tab, lin, n_dev, n_max, h->in_dim, (float*)feats);
        else if (out_dtype == NIF_BF16) k_encode_cat<float, __nv_bfloat16><<<g, 256, 0, s>>>(h->grid, tab, lin, n_dev, n_max, h->in_dim, (__nv_bfloat16*)feats);
        else k_encode_cat<float, __half><<<g, 256, 0, s>>>(h->grid, tab, lin, n_dev, n_max, h->in_dim, (__half*)feats);
    }
    NIF_CK_LAUNCH(h);
    return NIF_OK;
}

nif_status nif_encode_segments_run(nif_handle* h, const nif_linseg* lin, const uint32_t* n_dev, int64_t n_max,
                                   void* feats, int out_dtype, int table_dtype, cudaStream_t s, bool reuse_points,
                                   bool dedup) {
    NifProf prof_(h, "encode_fwd", s);
    if (n_max <= 0) return NIF_OK;
    nif_status st = NIF_OK;
    if (h->concat) return launch_cat(h, lin, n_dev, n_max, feats, out_dtype, table_dtype, s);
    if (table_dtype == NIF_FP16) {
        st = nif_refresh_lowp(h, s);
        if (st != NIF_OK) return st;
        const __half* tab = h->d_tables_h;
        if (out_dtype == NIF_FP32) st = launch_segments<__half, float>(h, tab, lin, n_dev, n_max, feats, s, reuse_points, dedup);
        else if (out_dtype == NIF_BF16) st = launch_segments<__half, __nv_bfloat16>(h, tab, lin, n_dev, n_max, feats, s, reuse_points, dedup);
        else if (out_dtype == NIF_FP16) st = launch_segments<__half, __half>(h, tab, lin, n_dev, n_max, feats, s, reuse_points, dedup);
        else return nif_fail(h, NIF_ERR_ARG, "out_dtype");
    } else if (table_dtype == NIF_FP32) {
        const float* tab = h->d_params + h->off_tables;
        if (out_dtype == NIF_FP32) st = launch_segments<float, float>(h, tab, lin, n_dev, n_max, feats, s, reuse_points, dedup);
        else if (out_dtype == NIF_BF16) st = launch_segments<float, __nv_bfloat16>(h, tab, lin, n_dev, n_max, feats, s, reuse_points, dedup);
        else if (out_dtype == NIF_FP16) st = launch_segments<float, __half>(h, tab, lin, n_dev, n_max, feats, s, reuse_points, dedup);
        else return nif_fail(h, NIF_ERR_ARG, "out_dtype");
    } else {
        return nif_fail(h, NIF_ERR_ARG, "table_dtype");
    }
    if (st != NIF_OK) return st;
    NIF_CK_LAUNCH(h);
    return NIF_OK;
}

nif_status nif_encode_points_bwd_run(nif_handle* h, const float* pts, int64_t n, const float* dfeats,
                                     float* dtables, float* dpts, cudaStream_t s) {
    NifProf prof_(h, "encode_points_bwd", s);
    if (n <= 0) return NIF_OK;
    if (h->concat) return nif_fail(h, NIF_ERR_ARG, "point encoding is the composed reading; this handle concatenates");
    if (dpts) NIF_CK(h, cudaMemsetAsync(dpts, 0, sizeof(float) * 3 * n, s));
    k_encode_points_bwd<<<nif_blocks(n * h->P, 256), 256, 0, s>>>(h->grid, h->d_params + h->off_tables, pts, n,
                                                                 dfeats, dtables, dpts);
    NIF_CK_LAUNCH(h);
    return NIF_OK;
}

// Deterministic mode's table gradient (see k_encode_bwd_fixed): the scale from
// max |dL/dfeature|, the fixed-point sums, their conversion into dtables.
// Level halves per task of the run-length backward (NIF_KNOB_BWD_SPLIT), where
// each half still holds the 3 lanes that evaluate a term's u.
// 0 (default) splits handles of L >= 16 (measured on the 64^3 FP32 step, L = 16:
// 2.77 ms against 2.83 ms, the backward 1.11 against 1.18 ms; the BF16 mixed and
// deterministic steps alike either way). With L = 8 a half holds 4 levels and a
// warp 8 terms, so the last term group would cut its chunk into 8 short runs.
static int bwd_split(const nif_handle* h) {
    const int k = h->tune.bwd_split == 0 ? (h->L >= 16 ? 2 : 1) : h->tune.bwd_split;
    return (k == 2 && h->L % 2 == 0 && 32 % (h->L / 2) == 0 && h->L / 2 >= 4) ? 2 : 1;
}

// The distinct end points the backward walks: the forward's list when it is
// of these segments (a training step), else listed (and ordered) here.
static nif_status bwd_points(nif_handle* h, const nif_linseg* lin, const uint32_t* n_dev, int64_t n_max,
                             bool reuse_points, const uint32_t** pts, const uint32_t** n_pts, const uint32_t** dupf,
                             cudaStream_t s) {
    // rest-space order: a lane's run of points stays in one small region,
    // so its cell cache flushes less at the middle levels
    const bool sorted = (size_t)h->T * h->L * h->Fd * sizeof(float) > ((size_t)4 << 20);
    const nif_handle::PointList& pl = h->enc_points;
    if (reuse_points && pl.pts && pl.lin == lin && pl.n_dev == n_dev && pl.n_max == n_max && pl.sorted == sorted) {
        *pts = pl.pts;                                    // as the forward of this step left them
        *n_pts = pl.n_pts;
        *dupf = pl.dupf;
        return NIF_OK;
    }
    nif_status st = distinct_points(h, lin, n_dev, n_max, pts, n_pts, dupf, s);
    if (st != NIF_OK) return st;
    if (sorted && (st = spatial_order(h, lin, *pts, *n_pts, n_max, pts, s)) != NIF_OK) return st;
    return NIF_OK;
}

// Dense prefix of levels of at most max_rows rows each that fits `budget`
// elements of shared memory (two per row).
static Coarse coarse_levels(const nif_handle* h, int64_t max_rows, int budget) {
    Coarse cs{};
    cs.Lc = 0;
    cs.soff[0] = 0;
    for (int l = 0; l < h->L; l++) {
        if (!((h->grid.dense_mask >> l) & 1u)) break;
        const int64_t r = (int64_t)h->grid.res[l] + 1;
        if (r * r * r > max_rows || cs.soff[l] + 2 * r * r * r > budget) break;
        cs.soff[l + 1] = cs.soff[l] + (int)(2 * r * r * r);
        cs.Lc = l + 1;
    }
    return cs;
}

// Deterministic mode's table gradient: the scale from max |dL/dfeature|
// (k_absmax_bits, k_fix_scale), the fixed-point sums -- by the run-length
// walk over the distinct points in their fixed order where the default path
// takes it (its per-cell FP32 sums depend only on the chunk's points and
// order, which are fixed, and are rounded once each), else one thread per
// (segment, end point, gamma term) -- and their conversion into dtables.
static nif_status encode_bwd_fixed(nif_handle* h, const nif_linseg* lin, const uint32_t* n_dev, int64_t n_max,
                                   const float* dfeats, float* dtables, cudaStream_t s, bool reuse_points, int ctas) {
    const int64_t cnt = (int64_t)h->L * h->T * 2;
    const size_t bytes = sizeof(unsigned long long) * (size_t)cnt;
    if (h->b_fix.bytes < bytes + 16) {
        nif_status st = nif_grow(h, h->b_fix, bytes + 16);
        if (st != NIF_OK) return st;
        NIF_CK(h, cudaMemsetAsync(h->b_fix.p, 0, bytes, s));      // zero between calls from here on
    }
    unsigned long long* fix = (unsigned long long*)h->b_fix.p;
    uint32_t* bits = (uint32_t*)((char*)h->b_fix.p + bytes);
    int* S_dev = (int*)(bits + 1);
    NIF_CK(h, cudaMemsetAsync(bits, 0, sizeof(uint32_t), s));
    const int64_t per = 4LL * h->P * h->L;                         // floats of dL/dfeature per segment
    const unsigned g4 = (unsigned)std::min<int64_t>(nif_blocks(n_max * per / 4, 256), (int64_t)h->num_sms * 8);
    k_absmax_bits<<<g4, 256, 0, s>>>(dfeats, n_dev, n_max, per, bits);
    NIF_CK_LAUNCH(h);
    k_fix_scale<<<1, 32, 0, s>>>(bits, n_dev, n_max, h->P, S_dev);
    NIF_CK_LAUNCH(h);
    if (32 % h->L == 0 && h->L >= 4) {
        const uint32_t *pts, *n_pts, *dupf;
        nif_status st = bwd_points(h, lin, n_dev, n_max, reuse_points, &pts, &n_pts, &dupf, s);
        if (st != NIF_OK) return st;
        const Coarse cs = coarse_levels(h, h->tune.bwd_smem_rows, 200 * 1024 / 8);
        const size_t smem = sizeof(unsigned long long) * (size_t)cs.soff[cs.Lc];
        auto kern = bwd_split(h) == 2 ? k_encode_segments_bwd_rl<true, 2> : k_encode_segments_bwd_rl<true, 1>;
        NIF_CK(h, cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
        NIF_CK(h, cudaMemsetAsync(h->d_next + 1, 0, sizeof(uint32_t), s));
        kern<<<ctas > 0 ? std::min(ctas, h->num_sms) : h->num_sms, 1024, smem, s>>>(
            h->grid, cs, lin, n_dev, n_max, dfeats, dtables, pts, n_pts, dupf, h->d_next + 1, fix, S_dev);
        NIF_CK_LAUNCH(h);
    } else {
        // dense coarse levels of at most 4096 rows in shared memory (96 KB at
        // most, two 1024-thread blocks per SM)
        const Coarse cs = coarse_levels(h, 4096, 96 * 1024 / 8);
        const size_t smem = sizeof(unsigned long long) * (size_t)cs.soff[cs.Lc];
        NIF_CK(h, cudaFuncSetAttribute(k_encode_bwd_fixed, cudaFuncAttributeMaxDynamicSharedMemorySize, 96 * 1024));
        const unsigned gb = (unsigned)std::min<int64_t>(nif_blocks(n_max * 2 * h->P, 1024), (int64_t)h->num_sms * 2);
        k_encode_bwd_fixed<<<gb, 1024, smem, s>>>(h->grid, cs, lin, n_dev, n_max, dfeats, fix, S_dev);
        NIF_CK_LAUNCH(h);
    }
    const unsigned gc = (unsigned)std::min<int64_t>(nif_blocks(cnt, 256), (int64_t)h->num_sms * 8);
    k_fix_to_float<<<gc, 256, 0, s>>>(fix, cnt, S_dev, dtables);
    NIF_CK_LAUNCH(h);
    return NIF_OK;
}

nif_status nif_encode_segments_bwd_run(nif_handle* h, const nif_linseg* lin, const uint32_t* n_dev, int64_t n_max,
                                       const float* dfeats, float* dtables, cudaStream_t s, bool reuse_points,
                                       int ctas) {
    NifProf prof_(h, "encode_bwd", s);
    if (n_max <= 0) return NIF_OK;
    if (h->det && !h->concat) return encode_bwd_fixed(h, lin, n_dev, n_max, dfeats, dtables, s, reuse_points, ctas);
    if (h->concat) {
        const int64_t work = n_max * 2 * h->L;
        k_encode_cat_bwd<<<(unsigned)std::min<int64_t>(nif_blocks(work, 256), (int64_t)h->num_sms * 16), 256, 0, s>>>(
            h->grid, lin, n_dev, n_max, h->in_dim, dfeats, dtables);
        NIF_CK_LAUNCH(h);
        return NIF_OK;
    }
    // dense prefix of levels that fits the shared-memory budget
    const Coarse cs = coarse_levels(h, h->tune.bwd_smem_rows, 200 * 1024 / 4);
    size_t smem = sizeof(float) * (size_t)cs.soff[cs.Lc];
    if (32 % h->L == 0 && h->L >= 4) {      // a level group holds the 3 lanes that evaluate u
        const uint32_t *pts, *n_pts, *dupf;
        nif_status st = bwd_points(h, lin, n_dev, n_max, reuse_points, &pts, &n_pts, &dupf, s);
        if (st != NIF_OK) return st;
        auto kern = bwd_split(h) == 2 ? k_encode_segments_bwd_rl<false, 2> : k_encode_segments_bwd_rl<false, 1>;
        NIF_CK(h, cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
        // at most one 1024-thread block per SM (64 registers a thread fill the
        // register file); its warps take chunks from the task counter
        NIF_CK(h, cudaMemsetAsync(h->d_next + 1, 0, sizeof(uint32_t), s));
        kern<<<ctas > 0 ? std::min(ctas, h->num_sms) : h->num_sms, 1024, smem, s>>>(
            h->grid, cs, lin, n_dev, n_max, dfeats, dtables, pts, n_pts, dupf, h->d_next + 1, nullptr, nullptr);
        NIF_CK_LAUNCH(h);
        return NIF_OK;
    }
    if (cs.Lc > 0) {
        NIF_CK(h, cudaFuncSetAttribute(k_encode_segments_bwd_sm, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       200 * 1024));
        k_encode_segments_bwd_sm<<<h->num_sms, 1024, smem, s>>>(h->grid, cs, lin, n_dev, n_max, dfeats, dtables);
        NIF_CK_LAUNCH(h);
        return NIF_OK;
    }
    unsigned g = nif_blocks(n_max * 2 * h->P, 256);
    unsigned cap = (unsigned)h->num_sms * 16;
    if (g > cap) g = cap;
    k_encode_segments_bwd<<<g, 256, 0, s>>>(h->grid, h->d_params + h->off_tables, lin, n_dev, n_max, dfeats,
                                            dtables);
    NIF_CK_LAUNCH(h);
    return NIF_OK;
}

nif_status nif_encode_segments_dp_run(nif_handle* h, const nif_linseg* lin, const uint32_t* n_dev, int64_t n,
                                      const float* dfeats, float* dp, cudaStream_t s) {
    NifProf prof_(h, "encode_dp", s);
    if (n <= 0) return NIF_OK;
    NIF_CK(h, cudaMemsetAsync(dp, 0, sizeof(float) * 6 * n, s));
    if (h->concat) {
        k_encode_cat_dp<<<(unsigned)std::min<int64_t>(nif_blocks(2 * n, 256), (int64_t)h->num_sms * 16), 256, 0, s>>>(
            h->grid, h->d_params + h->off_tables, lin, n_dev, n, h->in_dim, dfeats, dp);
        NIF_CK_LAUNCH(h);
        return NIF_OK;
    }
    unsigned g = nif_blocks(n * 2 * h->P, 256);
    unsigned cap = (unsigned)h->num_sms * 16;
    if (g > cap) g = cap;
    k_encode_segments_dp<<<g, 256, 0, s>>>(h->grid, h->d_params + h->off_tables, lin, n_dev, n, dfeats, dp);
    NIF_CK_LAUNCH(h);
    return NIF_OK;
}
