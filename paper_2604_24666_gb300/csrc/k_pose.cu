// k_pose.cu -- gradient of a loss with respect to the deformation parameters
// (pose fitting). A segment's rest end points are p = D^-1(x; theta) of fixed
// deformed points x, so D(p(theta); theta) = x and, by the implicit function
// theorem, dp/dtheta = -J_D(p)^-1 dD/dtheta(p). Given dL/dp of both end
// points, each segment contributes -(J_D^-T dL/dp) . dD/dtheta_j to
// dL/dtheta_j of its instance.
//
// With a learned deformation field (the paper's future work, Sec. 4; our
// reading: D = D_pose o (I + u), u trilinear over a lattice of displacements
// delta_n) the pose acts at q = p + u(p) with dL/dq = (I + du/dp)^-T dL/dp,
// and, q being fixed by x, p + u(p) = q gives dp/d(delta_n) = -(I + du/dp)^-1
// w_n(p): each end point adds -w_n(p) (I + du/dp)^-T dL/dp to the gradient of
// node n of its instance's field.
#include <cmath>
#include <vector>

#include "nif_internal.cuh"

namespace {

__device__ __forceinline__ int find_inst_p(const int* inst_off, int n_inst, int r) {
    if (!inst_off || n_inst <= 1) return 0;
    int lo = 0, hi = n_inst - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (__ldg(inst_off + mid) <= r) lo = mid; else hi = mid - 1;
    }
    return lo;
}

__global__ void __launch_bounds__(256) k_pose_grad(const nif_segment* __restrict__ segs,
                                                   const nif_linseg* __restrict__ lin, const float* __restrict__ dp,
                                                   const uint32_t* __restrict__ n_dev, int64_t n_max,
                                                   const int* __restrict__ inst_off, int n_inst,
                                                   const float4* __restrict__ poses, FieldView f,
                                                   float* __restrict__ dposes) {
    int64_t n = n_dev ? (int64_t)*n_dev : n_max;
    if (n > n_max) n = n_max;
    for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < n; s += (int64_t)gridDim.x * blockDim.x) {
        int inst = find_inst_p(inst_off, n_inst, (int)segs[s].ray);
        float4 pose = poses[inst];
        float g0 = 0.f, g1 = 0.f, g2 = 0.f;
        for (int e = 0; e < 2; e++) {
            const float* P = reinterpret_cast<const float*>(lin + s) + 3 * e;
            float3 p = make_float3(P[0], P[1], P[2]);
            float3 d = make_float3(dp[s * 6 + e * 3], dp[s * 6 + e * 3 + 1], dp[s * 6 + e * 3 + 2]);
            if (f.d && inst < f.n) {        // to q = p + u(p), where the pose acts
                float3 g[3];
                const float3 u = nif_field_eval(f, inst, p, g);
                d = nif_solve3_t(make_float3(1.f + g[0].x, g[0].y, g[0].z), make_float3(g[1].x, 1.f + g[1].y, g[1].z),
                                 make_float3(g[2].x, g[2].y, 1.f + g[2].z), d);
                p = make_float3(p.x + u.x, p.y + u.y, p.z + u.z);
            }
            float3 j0, j1, j2;
            nif_jacobian_cols(p, pose, j0, j1, j2);
            float3 c0 = nif_cross(j1, j2), c1 = nif_cross(j2, j0), c2 = nif_cross(j0, j1);
            float det = j0.x * c0.x + j0.y * c0.y + j0.z * c0.z;
            float id = 1.0f / det;
            // y = J^-T dL/dp
            float3 y = make_float3((d.x * c0.x + d.y * c1.x + d.z * c2.x) * id,
                                   (d.x * c0.y + d.y * c1.y + d.z * c2.y) * id,
                                   (d.x * c0.z + d.y * c1.z + d.z * c2.z) * id);
            float3 dk, dth, dta;
            nif_param_jacobian_cols(p, pose, dk, dth, dta);
            g0 -= NIF_KBEND * (y.x * dk.x + y.y * dk.y + y.z * dk.z);
            g1 -= y.x * dth.x + y.y * dth.y + y.z * dth.z;
            g2 -= y.x * dta.x + y.y * dta.y + y.z * dta.z;
        }
        // reduce over the warp when it is complete and all its segments belong
        // to one instance; otherwise every lane adds its own contribution
        unsigned m = __activemask();
        bool uniform = false;
        if (m == 0xffffffffu) {
            int inst0 = __shfl_sync(m, inst, 0);
            uniform = __all_sync(m, inst == inst0);
        }
        if (uniform) {
            for (int o = 16; o > 0; o >>= 1) {
                g0 += __shfl_down_sync(m, g0, o);
                g1 += __shfl_down_sync(m, g1, o);
                g2 += __shfl_down_sync(m, g2, o);
            }
            if ((threadIdx.x & 31) == 0) {
                atomicAdd(dposes + 3 * inst, g0);
                atomicAdd(dposes + 3 * inst + 1, g1);
                atomicAdd(dposes + 3 * inst + 2, g2);
            }
        } else {
            atomicAdd(dposes + 3 * inst, g0);
            atomicAdd(dposes + 3 * inst + 1, g1);
            atomicAdd(dposes + 3 * inst + 2, g2);
        }
    }
}

// Field gradient: one thread per segment, both end points; the block's
// share is summed in shared memory (the lattice is small and every point
// touches 8 nodes) and added to global memory once per block, when it fits
// (smem_nodes > 0); otherwise every contribution is a global atomic.
__global__ void __launch_bounds__(256) k_field_grad(const nif_segment* __restrict__ segs,
                                                    const nif_linseg* __restrict__ lin, const float* __restrict__ dp,
                                                    const uint32_t* __restrict__ n_dev, int64_t n_max,
                                                    const int* __restrict__ inst_off, int n_inst, FieldView f,
                                                    int smem_nodes, float* __restrict__ dfield) {
    extern __shared__ float acc[];
    const int G3 = f.G * f.G * f.G;
    for (int i = threadIdx.x; i < 3 * smem_nodes; i += blockDim.x) acc[i] = 0.f;
    __syncthreads();
    int64_t n = n_dev ? (int64_t)*n_dev : n_max;
    if (n > n_max) n = n_max;
    for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < n; s += (int64_t)gridDim.x * blockDim.x) {
        const int inst = find_inst_p(inst_off, n_inst, (int)segs[s].ray);
        if (inst >= f.n) continue;
        for (int e = 0; e < 2; e++) {
            const float* P = reinterpret_cast<const float*>(lin + s) + 3 * e;
            const float3 p = make_float3(P[0], P[1], P[2]);
            const float3 d = make_float3(dp[s * 6 + e * 3], dp[s * 6 + e * 3 + 1], dp[s * 6 + e * 3 + 2]);
            float3 g[3];
            nif_field_eval(f, inst, p, g);
            const float3 v = nif_solve3_t(make_float3(1.f + g[0].x, g[0].y, g[0].z),
                                          make_float3(g[1].x, 1.f + g[1].y, g[1].z),
                                          make_float3(g[2].x, g[2].y, 1.f + g[2].z), d);
            int i, j, k;
            float3 t;
            nif_field_cell(f.G, p, i, j, k, t);
#pragma unroll
            for (int c = 0; c < 8; c++) {
                const int a = c & 1, b = (c >> 1) & 1, cc = (c >> 2) & 1;
                const float w = (a ? t.x : 1.f - t.x) * (b ? t.y : 1.f - t.y) * (cc ? t.z : 1.f - t.z);
                const int node = inst * G3 + ((k + cc) * f.G + (j + b)) * f.G + (i + a);
                float* dst = node < smem_nodes ? acc + 3 * node : dfield + 3 * (int64_t)node;
                atomicAdd(dst, -w * v.x);
                atomicAdd(dst + 1, -w * v.y);
                atomicAdd(dst + 2, -w * v.z);
            }
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < 3 * smem_nodes; i += blockDim.x)
        if (acc[i] != 0.f) atomicAdd(dfield + i, acc[i]);
}

// Adam on the field's displacements (moments in the field's float4 layout),
// the gradient [n][G^3][3] cleared after use
__global__ void k_field_adam(float4* __restrict__ d, float4* __restrict__ m, float4* __restrict__ v,
                             float* __restrict__ g, int64_t nodes, float lr, float c1, float c2) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nodes; i += (int64_t)gridDim.x * blockDim.x) {
        float* gi = g + 3 * i;
        float4 di = d[i], mi = m[i], vi = v[i];
        float* dd = &di.x;
        float* mm = &mi.x;
        float* vv = &vi.x;
#pragma unroll
        for (int c = 0; c < 3; c++) {
            const float gr = gi[c];
            mm[c] = 0.9f * mm[c] + 0.1f * gr;
            vv[c] = 0.99f * vv[c] + 0.01f * gr * gr;
            dd[c] -= lr * (mm[c] * c1) / (sqrtf(vv[c] * c2) + 1e-15f);
            gi[c] = 0.f;
        }
        d[i] = di;
        m[i] = mi;
        v[i] = vi;
    }
}

// The field's Lipschitz bound, per instance (as the oracle's field_lipschitz):
// within a cell, du/dp_a is a convex combination of its four edge differences
// along a times (G-1), so |du/dp|_2 <= sqrt(sum_a ((G-1) max_edge_a |delta_b -
// delta_a|)^2). One thread per cell; the maximum over cells by an atomic max
// on the (non-negative) float's bits.
__global__ void k_field_lipschitz(const float4* __restrict__ d, int G, int n_inst, float* __restrict__ lip) {
    const int C = G - 1;
    const int64_t cells = (int64_t)C * C * C;
    for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < cells * n_inst;
         x += (int64_t)gridDim.x * blockDim.x) {
        const int inst = (int)(x / cells);
        const int64_t c = x - (int64_t)inst * cells;
        const int i = (int)(c % C), j = (int)((c / C) % C), k = (int)(c / ((int64_t)C * C));
        const float4* D = d + (int64_t)inst * G * G * G;
        auto at = [&](int a, int b, int e) { return __ldg(D + ((int64_t)(k + e) * G + (j + b)) * G + (i + a)); };
        auto dist = [](float4 p, float4 q) {
            const float dx = p.x - q.x, dy = p.y - q.y, dz = p.z - q.z;
            return sqrtf(dx * dx + dy * dy + dz * dz);
        };
        float ex = 0.f, ey = 0.f, ez = 0.f;
        for (int u = 0; u < 2; u++)
            for (int w = 0; w < 2; w++) {
                ex = fmaxf(ex, dist(at(1, u, w), at(0, u, w)));
                ey = fmaxf(ey, dist(at(u, 1, w), at(u, 0, w)));
                ez = fmaxf(ez, dist(at(u, w, 1), at(u, w, 0)));
            }
        const float l = (float)C * sqrtf(ex * ex + ey * ey + ez * ez);
        atomicMax(reinterpret_cast<unsigned int*>(lip + inst), __float_as_uint(l));
    }
}

// An instance's field whose bound passed `bound` is scaled back onto it (the
// bound is homogeneous of degree one in the displacements)
__global__ void k_field_project(float4* __restrict__ d, int G3, int n_inst, const float* __restrict__ lip,
                                float bound) {
    const int64_t total = (int64_t)G3 * n_inst;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
        const float l = lip[i / G3];
        if (l > bound) {
            const float sc = bound / l;
            float4 v = d[i];
            d[i] = make_float4(v.x * sc, v.y * sc, v.z * sc, 0.f);
        }
    }
}

}  // namespace

nif_status nif_field_grad_run(nif_handle* h, const nif_segment* segs, const nif_linseg* lin, const float* dp,
                              const uint32_t* n_dev, int64_t n, const int* inst_off, int n_inst, float* dfield,
                              cudaStream_t s) {
    NifProf prof_(h, "field_grad", s);
    if (n <= 0 || h->field_G == 0) return NIF_OK;
    const FieldView f = nif_field_view(h);
    const int64_t nodes = (int64_t)f.G * f.G * f.G * std::min(n_inst, f.n);
    const int smem_nodes = 3 * nodes * (int64_t)sizeof(float) <= 48 * 1024 ? (int)nodes : 0;
    unsigned g = nif_blocks(n, 256);
    unsigned cap = (unsigned)h->num_sms * 2;
    if (g > cap) g = cap;
    k_field_grad<<<g, 256, sizeof(float) * 3 * smem_nodes, s>>>(segs, lin, dp, n_dev, n, inst_off, n_inst, f,
                                                                smem_nodes, dfield);
    NIF_CK_LAUNCH(h);
    return NIF_OK;
}

nif_status nif_field_adam_run(nif_handle* h, float lr, cudaStream_t s) {
    NifProf prof_(h, "field_adam", s);
    if (h->field_G == 0) return NIF_OK;
    const int G3 = h->field_G * h->field_G * h->field_G;
    const int64_t nodes = (int64_t)G3 * h->field_n;
    h->field_step++;
    const double b1t = std::pow(0.9, (double)h->field_step), b2t = std::pow(0.99, (double)h->field_step);
    const unsigned g = std::min<unsigned>(nif_blocks(nodes, 256), (unsigned)h->num_sms * 4);
    k_field_adam<<<g, 256, 0, s>>>(h->d_field, h->d_field_m, h->d_field_v, h->d_field_g, nodes, lr,
                                   (float)(1.0 / (1.0 - b1t)), (float)(1.0 / (1.0 - b2t)));
    NIF_CK_LAUNCH(h);
    NIF_CK(h, cudaMemsetAsync(h->d_field_lip, 0, sizeof(float) * h->field_n, s));
    const int64_t cells = (int64_t)(h->field_G - 1) * (h->field_G - 1) * (h->field_G - 1) * h->field_n;
    k_field_lipschitz<<<std::min<unsigned>(nif_blocks(cells, 256), (unsigned)h->num_sms * 4), 256, 0, s>>>(
        h->d_field, h->field_G, h->field_n, h->d_field_lip);
    NIF_CK_LAUNCH(h);
    k_field_project<<<g, 256, 0, s>>>(h->d_field, G3, h->field_n, h->d_field_lip, NIF_FIELD_MAX_LIPSCHITZ);
    NIF_CK_LAUNCH(h);
    return NIF_OK;
}

nif_status nif_pose_grad_run(nif_handle* h, const nif_segment* segs, const nif_linseg* lin, const float* dp,
                             const uint32_t* n_dev, int64_t n, const int* inst_off, int n_inst, float* dposes,
                             cudaStream_t s) {
    NifProf prof_(h, "pose_grad", s);
    if (n <= 0) return NIF_OK;
    unsigned g = nif_blocks(n, 256);
    unsigned cap = (unsigned)h->num_sms * 8;
    if (g > cap) g = cap;
    k_pose_grad<<<g, 256, 0, s>>>(segs, lin, dp, n_dev, n, inst_off, n_inst, h->d_pose, nif_field_view(h), dposes);
    NIF_CK_LAUNCH(h);
    return NIF_OK;
}
