// enc_grid.cuh -- device building blocks of the hybrid encoding psi = phi o
// gamma (Eq. 1) shared by the encoding kernels (k_encode.cu) and the fused
// encoding + tensor-core MLP of the query path (k_mlp_enc.cu): the cell and
// trilinear weights of a level, the u of a gamma term, and the gather of a
// level's 8 corner rows (dense index or spatial hash).
#pragma once

#include "nif_internal.cuh"

namespace {

struct Cell {
    int ix, iy, iz;
    float wx, wy, wz;
};

__device__ __forceinline__ Cell cell_of(float3 u, int Nl) {
    float fn = (float)Nl;
    float qx = __fmul_rn(u.x, fn), qy = __fmul_rn(u.y, fn), qz = __fmul_rn(u.z, fn);
    Cell c;
    c.ix = min((int)floorf(qx), Nl - 1);
    c.iy = min((int)floorf(qy), Nl - 1);
    c.iz = min((int)floorf(qz), Nl - 1);
    // bounds build: a cell outside the level's grid would put corner rows
    // past the level's block; it is counted and the cell moved to the origin
    if (!(NIF_IN(c.ix, Nl) && NIF_IN(c.iy, Nl) && NIF_IN(c.iz, Nl))) c.ix = c.iy = c.iz = 0;
    c.wx = qx - (float)c.ix;
    c.wy = qy - (float)c.iy;
    c.wz = qz - (float)c.iz;
    return c;
}

// u of term t of gamma(p); p already clamped to [0,1]
__device__ __forceinline__ float3 term_u(float3 p, int t) {
    if (t == 0) return p;
    int k = (t - 1) >> 1;
    float f = (float)(1 << k);
    float sx, cx, sy, cy, sz, cz;
    sincosf(f * p.x, &sx, &cx);
    sincosf(f * p.y, &sy, &cy);
    sincosf(f * p.z, &sz, &cz);
    if ((t - 1) & 1) return make_float3((cx + 1.0f) * 0.5f, (cy + 1.0f) * 0.5f, (cz + 1.0f) * 0.5f);
    return make_float3((sx + 1.0f) * 0.5f, (sy + 1.0f) * 0.5f, (sz + 1.0f) * 0.5f);
}

__device__ __forceinline__ float3 clamp01(float3 p) {
    return make_float3(fminf(fmaxf(p.x, 0.f), 1.f), fminf(fmaxf(p.y, 0.f), 1.f), fminf(fmaxf(p.z, 0.f), 1.f));
}

// a table row as loaded (two FP32 or two FP16 features), converted at use
template <typename TT>
struct RawRow;
template <>
struct RawRow<float> {
    using T = float2;
    static __device__ __forceinline__ T load(const float* tab, uint32_t row) {
        return __ldg(reinterpret_cast<const float2*>(tab) + row);
    }
    static __device__ __forceinline__ float2 f2(T v) { return v; }
};
template <>
struct RawRow<__half> {
    using T = __half2;
    static __device__ __forceinline__ T load(const __half* tab, uint32_t row) {
        return __ldg(reinterpret_cast<const __half2*>(tab) + row);
    }
    static __device__ __forceinline__ float2 f2(T v) { return __half22float2(v); }
};

// the 8 corner rows of level l's cell c (dense index or spatial hash), loaded
template <typename TT>
__device__ __forceinline__ void level_gather(const GridInfo& g, const TT* __restrict__ tab, int l, const Cell& c,
                                             typename RawRow<TT>::T* v) {
    const int Nl = g.res[l];
    const TT* tl = tab + (int64_t)l * g.T * 2;
    uint32_t rows[8];
    if ((g.dense_mask >> l) & 1u) {
        const uint32_t sy = (uint32_t)Nl + 1u, sz = sy * sy;
        const uint32_t b = (uint32_t)c.ix + (uint32_t)c.iy * sy + (uint32_t)c.iz * sz;
        rows[0] = b; rows[1] = b + 1u; rows[2] = b + sy; rows[3] = b + sy + 1u;
        rows[4] = b + sz; rows[5] = b + sz + 1u; rows[6] = b + sz + sy; rows[7] = b + sz + sy + 1u;
    } else {
        const uint32_t m = g.T - 1u;
        const uint32_t x0 = (uint32_t)c.ix, x1 = x0 + 1u;
        const uint32_t y0 = (uint32_t)c.iy * 2654435761u, y1 = y0 + 2654435761u;
        const uint32_t z0 = (uint32_t)c.iz * 805459861u, z1 = z0 + 805459861u;
        rows[0] = (x0 ^ y0 ^ z0) & m; rows[1] = (x1 ^ y0 ^ z0) & m;
        rows[2] = (x0 ^ y1 ^ z0) & m; rows[3] = (x1 ^ y1 ^ z0) & m;
        rows[4] = (x0 ^ y0 ^ z1) & m; rows[5] = (x1 ^ y0 ^ z1) & m;
        rows[6] = (x0 ^ y1 ^ z1) & m; rows[7] = (x1 ^ y1 ^ z1) & m;
    }
#pragma unroll
    for (int q = 0; q < 8; q++) v[q] = RawRow<TT>::load(tl, rows[q]);
}

}  // namespace
