// k_train.cu -- ground-truth labels of linearized segments (Sec. 2), task
// losses with uncertainty weighting (Sec. 2.4), Adam, the segmented-ray
// reconstruction (Sec. 2.2) and the counter-based sampler of training rays.
#include <algorithm>

#include "nif_internal.cuh"

namespace {

// ---------------------------------------------------------------------------
// Labels: straight rest segment p0 -> p1 against the voxel's triangles
// (Moeller-Trumbore, FP32); first hit in [0,1], ties to the smaller id.
// ---------------------------------------------------------------------------
// One record per triangle for the labels: A, e1 = B - A, e2 = C - A, each
// difference the FP32 subtraction the test would do, read as 3 float4 in
// place of 3 vertex indices and 9 dependent vertex loads.
__global__ void __launch_bounds__(256) k_tri_geo(const float* __restrict__ verts, const int* __restrict__ tris,
                                                 int n_tris, float4* __restrict__ geo) {
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < n_tris; t += gridDim.x * blockDim.x) {
        const int i0 = tris[3 * t], i1 = tris[3 * t + 1], i2 = tris[3 * t + 2];
        const float Ax = verts[3 * i0], Ay = verts[3 * i0 + 1], Az = verts[3 * i0 + 2];
        const float e1x = verts[3 * i1] - Ax, e1y = verts[3 * i1 + 1] - Ay, e1z = verts[3 * i1 + 2] - Az;
        const float e2x = verts[3 * i2] - Ax, e2y = verts[3 * i2 + 1] - Ay, e2z = verts[3 * i2 + 2] - Az;
        geo[3 * t] = make_float4(Ax, Ay, Az, e1x);
        geo[3 * t + 1] = make_float4(e1y, e1z, e2x, e2y);
        geo[3 * t + 2] = make_float4(e2z, 0.f, 0.f, 0.f);
    }
}

__global__ void __launch_bounds__(256) k_labels(const nif_segment* __restrict__ segs,
                                                const nif_linseg* __restrict__ lin,
                                                const uint32_t* __restrict__ n_dev, int64_t n_max,
                                                const uint32_t* __restrict__ tri_ptr,
                                                const int32_t* __restrict__ tri_idx,
                                                const float4* __restrict__ geo,
                                                const float* __restrict__ alb, const uint8_t* __restrict__ mat,
                                                nif_label* __restrict__ out, int* __restrict__ n_hit,
                                                uint32_t nvox, int n_tris) {
    int64_t n = n_dev ? (int64_t)*n_dev : n_max;
    if (n > n_max) n = n_max;
    int local_hits = 0;
    for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < n; s += (int64_t)gridDim.x * blockDim.x) {
        const float* L = reinterpret_cast<const float*>(lin + s);
        float ox = L[0], oy = L[1], oz = L[2];
        float dx = L[3] - ox, dy = L[4] - oy, dz = L[5] - oz;
        uint32_t v = segs[s].voxel;
        uint32_t a = 0, b = 0;
        if (v < nvox) { a = tri_ptr[v]; b = tri_ptr[v + 1]; }    // foreign voxel ids label as empty
        float best = 2.0f;
        int bt = -1;
        for (uint32_t q = a; q < b; q++) {
            int t = tri_idx[q];
            if (!NIF_IN(t, n_tris)) continue;
            const float4 g0 = __ldg(geo + 3 * t), g1 = __ldg(geo + 3 * t + 1), g2 = __ldg(geo + 3 * t + 2);
            float Ax = g0.x, Ay = g0.y, Az = g0.z;
            float e1x = g0.w, e1y = g1.x, e1z = g1.y;
            float e2x = g1.z, e2y = g1.w, e2z = g2.x;
            float px = dy * e2z - dz * e2y, py = dz * e2x - dx * e2z, pz = dx * e2y - dy * e2x;
            float det = e1x * px + e1y * py + e1z * pz;
            if (det == 0.f) continue;
            float inv = 1.0f / det;
            float sx = ox - Ax, sy = oy - Ay, sz = oz - Az;
            float u = (sx * px + sy * py + sz * pz) * inv;
            if (u < 0.f || u > 1.f) continue;
            float qx = sy * e1z - sz * e1y, qy = sz * e1x - sx * e1z, qz = sx * e1y - sy * e1x;
            float w = (dx * qx + dy * qy + dz * qz) * inv;
            if (w < 0.f || u + w > 1.f) continue;
            float tt = (e2x * qx + e2y * qy + e2z * qz) * inv;
            if (tt < 0.f || tt > 1.f) continue;
            if (tt < best) { best = tt; bt = t; }
        }
        nif_label lab;
        if (bt < 0) {
            lab.tpar = 0.f;
            lab.normal[0] = lab.normal[1] = lab.normal[2] = 0.f;
            lab.albedo[0] = lab.albedo[1] = lab.albedo[2] = 0.f;
            lab.occ = 0;
            lab.material = 0;
        } else {
            const float4 g0 = __ldg(geo + 3 * bt), g1 = __ldg(geo + 3 * bt + 1), g2 = __ldg(geo + 3 * bt + 2);
            float e1x = g0.w, e1y = g1.x, e1z = g1.y;
            float e2x = g1.z, e2y = g1.w, e2z = g2.x;
            float nx = e1y * e2z - e1z * e2y, ny = e1z * e2x - e1x * e2z, nz = e1x * e2y - e1y * e2x;
            float il = rsqrtf(nx * nx + ny * ny + nz * nz);
            lab.tpar = best;
            lab.normal[0] = nx * il; lab.normal[1] = ny * il; lab.normal[2] = nz * il;
            lab.albedo[0] = alb[3 * bt]; lab.albedo[1] = alb[3 * bt + 1]; lab.albedo[2] = alb[3 * bt + 2];
            lab.occ = 1;
            lab.material = mat[bt];
            local_hits++;
        }
        lab.pad[0] = lab.pad[1] = 0;
        out[s] = lab;
    }
    if (n_hit) {
        for (int o = 16; o > 0; o >>= 1) local_hits += __shfl_down_sync(0xffffffffu, local_hits, o);
        if ((threadIdx.x & 31) == 0 && local_hits) atomicAdd(n_hit, local_hits);
    }
}

// ---------------------------------------------------------------------------
// Loss (Sec. 2.4). acc[0..4] += sums of the five task losses.
// ---------------------------------------------------------------------------
__device__ __forceinline__ float sigmoidf_(float z) { return 1.0f / (1.0f + expf(-z)); }
__device__ __forceinline__ float softplusf_(float z) { return fmaxf(z, 0.f) + log1pf(expf(-fabsf(z))); }

__global__ void __launch_bounds__(256) k_loss(const float* __restrict__ out, const nif_label* __restrict__ labels,
                                              const nif_linseg* __restrict__ lin, const uint32_t* __restrict__ n_dev,
                                              int64_t n_max, const int* __restrict__ n_hit,
                                              const float* __restrict__ s_par, int N, int M, unsigned flags,
                                              float* __restrict__ dout, double* __restrict__ acc,
                                              double* __restrict__ parts) {
    int64_t n = n_dev ? (int64_t)*n_dev : n_max;
    if (n > n_max) n = n_max;
    int nh = *n_hit;
    float inv_h = nh > 0 ? 1.0f / (float)nh : 0.f;
    float inv_n = n > 0 ? 1.0f / (float)n : 0.f;
    float es[5];
    const bool fixed_w = flags & NIF_FLAG_FIXED_TASK_WEIGHTS;
    const bool sig_d = flags & NIF_FLAG_SIGMOID_DISTANCE;
#pragma unroll
    for (int i = 0; i < 5; i++) es[i] = fixed_w ? 1.0f : expf(-s_par[i]);
    float part[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
    for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < n; s += (int64_t)gridDim.x * blockDim.x) {
        const float* z = out + s * NIF_OUT;
        nif_label lab = labels[s];
        int mcls = lab.material < M ? lab.material : M - 1;
        float g[NIF_OUT];
#pragma unroll
        for (int i = 0; i < NIF_OUT; i++) g[i] = 0.f;
        // occlusion: BCE with logits over all segments
        float occ = lab.occ ? 1.f : 0.f;
        part[4] += softplusf_(z[0]) - occ * z[0];
        g[0] = (sigmoidf_(z[0]) - occ) * es[4] * inv_n;
        if (lab.occ) {
            float y = lab.tpar * lin[s].l_rest * (float)N;
            if (sig_d) {
                // ablation: bounded sigmoid head, squared error of the distance itself
                float sg = sigmoidf_(z[1]);
                float e = 1.7320508075688772f * sg - y;
                part[0] += e * e;
                g[1] = 0.5f * es[0] * 2.0f * e * 1.7320508075688772f * sg * (1.f - sg) * inv_h;
            } else {
                // distance: ReLU head, MSE of logs, target in voxel units
                float dh = fmaxf(z[1], 0.f);
                float e = logf(dh + NIF_EPS_DIST) - logf(y + NIF_EPS_DIST);
                part[0] += e * e;
                g[1] = z[1] > 0.f ? 0.5f * es[0] * 2.0f * e / (dh + NIF_EPS_DIST) * inv_h : 0.f;
            }
            // normal: 1 - cos
            float nx = z[2], ny = z[3], nz = z[4];
            float nn = fmaxf(sqrtf(nx * nx + ny * ny + nz * nz), 1e-8f);
            float dot = nx * lab.normal[0] + ny * lab.normal[1] + nz * lab.normal[2];
            part[1] += 1.0f - dot / nn;
            float c1 = -0.5f * es[1] * inv_h / nn, c2 = 0.5f * es[1] * inv_h * dot / (nn * nn * nn);
            g[2] = c1 * lab.normal[0] + c2 * nx;
            g[3] = c1 * lab.normal[1] + c2 * ny;
            g[4] = c1 * lab.normal[2] + c2 * nz;
            // albedo: sigmoid + L1
#pragma unroll
            for (int c = 0; c < 3; c++) {
                float a = sigmoidf_(z[5 + c]);
                float d = a - lab.albedo[c];
                part[2] += fabsf(d) * (1.0f / 3.0f);
                float sg = d > 0.f ? 1.f : (d < 0.f ? -1.f : 0.f);
                g[5 + c] = sg * a * (1.f - a) * 0.5f * es[2] * inv_h * (1.0f / 3.0f);
            }
            // material: cross entropy
            float mx = -3.0e38f;
            for (int c = 0; c < M; c++) mx = fmaxf(mx, z[8 + c]);
            float se = 0.f;
            for (int c = 0; c < M; c++) se += expf(z[8 + c] - mx);
            float lse = mx + logf(se);
            part[3] += lse - z[8 + mcls];
            for (int c = 0; c < M; c++) {
                float p = expf(z[8 + c] - lse);
                g[8 + c] = (p - (c == mcls ? 1.f : 0.f)) * es[3] * inv_h;
            }
        }
        if (dout) {
            float4* D4 = reinterpret_cast<float4*>(dout + s * NIF_OUT);
#pragma unroll
            for (int q = 0; q < NIF_OUT / 4; q++) D4[q] = make_float4(g[4 * q], g[4 * q + 1], g[4 * q + 2], g[4 * q + 3]);
        }
    }
    __shared__ float sh[8][5];
#pragma unroll
    for (int i = 0; i < 5; i++) {
        float v = part[i];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5][i] = v;
    }
    __syncthreads();
    if (threadIdx.x < 5) {
        double t = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); w++) t += sh[w][threadIdx.x];
        // deterministic mode: each block's sums are kept and added in block order
        if (parts) parts[5 * blockIdx.x + threadIdx.x] = t;
        else atomicAdd(acc + threadIdx.x, t);
    }
}

// parts -> total and dL/ds (added into the gradient buffer)
__global__ void k_loss_final(double* acc, const double* __restrict__ parts, int n_parts,
                             const uint32_t* __restrict__ n_dev, int64_t n_max,
                             const int* __restrict__ n_hit, const float* __restrict__ s_par, unsigned flags,
                             float* __restrict__ ds, int* status) {
    if (threadIdx.x != 0) return;
    if (parts)
        for (int i = 0; i < 5; i++) {
            double t = 0;
            for (int b = 0; b < n_parts; b++) t += parts[5 * b + i];
            acc[i] = t;
        }
    int64_t n = n_dev ? (int64_t)*n_dev : n_max;
    if (n > n_max) n = n_max;
    int nh = *n_hit;
    double L[5];
    for (int i = 0; i < 4; i++) L[i] = nh > 0 ? acc[i] / nh : 0.0;
    L[4] = n > 0 ? acc[4] / n : 0.0;
    const double wreg[5] = {0.5, 0.5, 0.5, 1.0, 1.0};
    double total = 0;
    const bool fixed_w = flags & NIF_FLAG_FIXED_TASK_WEIGHTS;
    for (int i = 0; i < 5; i++) {
        if (fixed_w) {
            total += wreg[i] * L[i];
            continue;
        }
        double es = exp(-(double)s_par[i]);
        total += wreg[i] * es * L[i] + 0.5 * s_par[i];
        if (ds) ds[i] += (float)(-wreg[i] * es * L[i] + 0.5);
    }
    acc[8] = total;
    for (int i = 0; i < 5; i++) acc[9 + i] = L[i];
    if (!isfinite(total)) nif_set_status(status, NIF_ERR_NAN);
}

// ---------------------------------------------------------------------------
// Adam over the whole parameter buffer; zeroes the gradient afterwards.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void adam_elem(float& p, float gi, float& m, float& v, float lr, float c1, float c2) {
    const float b1 = 0.9f, b2 = 0.99f, eps = 1e-15f;
    const float mi = b1 * m + (1.f - b1) * gi;
    const float vi = b2 * v + (1.f - b2) * gi * gi;
    m = mi;
    v = vi;
    p -= lr * (mi * c1) / (sqrtf(vi * c2) + eps);
}

// Four parameters a thread per iteration through 16-byte accesses (the four
// buffers come from cudaMalloc, so element 4j starts a 16-byte boundary),
// then the n % 4 tail one by one.
__global__ void __launch_bounds__(256) k_adam(float* __restrict__ p, float* __restrict__ g, float* __restrict__ m,
                                              float* __restrict__ v, size_t n, size_t mlp_begin, size_t mlp_end,
                                              float lr_grid, float lr_mlp, float c1, float c2) {
    const size_t stride = (size_t)gridDim.x * blockDim.x;
    const size_t tid = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    const size_t n4 = n / 4;
    for (size_t j = tid; j < n4; j += stride) {
        const float4 g4 = reinterpret_cast<const float4*>(g)[j];
        float4 p4 = reinterpret_cast<float4*>(p)[j];
        float4 m4 = reinterpret_cast<float4*>(m)[j];
        float4 v4 = reinterpret_cast<float4*>(v)[j];
        const size_t i = 4 * j;
        auto lr = [&](size_t k) { return (k >= mlp_begin && k < mlp_end) ? lr_mlp : lr_grid; };
        adam_elem(p4.x, g4.x, m4.x, v4.x, lr(i), c1, c2);
        adam_elem(p4.y, g4.y, m4.y, v4.y, lr(i + 1), c1, c2);
        adam_elem(p4.z, g4.z, m4.z, v4.z, lr(i + 2), c1, c2);
        adam_elem(p4.w, g4.w, m4.w, v4.w, lr(i + 3), c1, c2);
        reinterpret_cast<float4*>(m)[j] = m4;
        reinterpret_cast<float4*>(v)[j] = v4;
        reinterpret_cast<float4*>(p)[j] = p4;
        reinterpret_cast<float4*>(g)[j] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
    for (size_t i = 4 * n4 + tid; i < n; i += stride) {
        adam_elem(p[i], g[i], m[i], v[i], (i >= mlp_begin && i < mlp_end) ? lr_mlp : lr_grid, c1, c2);
        g[i] = 0.f;
    }
}

// ---------------------------------------------------------------------------
// Mixed-precision training: gradient check, Adam on the unscaled gradient
// with overflow skip, dynamic loss scale update.
// ---------------------------------------------------------------------------
constexpr float kScaleGrowth = 2.0f, kScaleBackoff = 0.5f;
constexpr int kScaleInterval = 2000;        // clean steps before S doubles
constexpr float kScaleMax = 16777216.0f, kScaleMin = 1.0f / 16384.0f;

__global__ void __launch_bounds__(256) k_grad_check(const float* __restrict__ g, size_t n, NifLossScale* ls) {
    bool bad = false;
    const size_t n4 = n / 4;
    const float4* g4 = reinterpret_cast<const float4*>(g);
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n4; i += (size_t)gridDim.x * blockDim.x) {
        float4 v = g4[i];
        bad |= !(isfinite(v.x) && isfinite(v.y) && isfinite(v.z) && isfinite(v.w));
    }
    for (size_t i = n4 * 4 + (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        bad |= !isfinite(g[i]);
    if (__syncthreads_or(bad) && threadIdx.x == 0) atomicExch(&ls->overflow, 1);
}

// Adam (same constants as k_adam) on g / S for [0, unscale_end) and g beyond
// (the task log-variances, whose gradient the loss writes unscaled); the whole
// step is skipped when the check found a non-finite gradient. Bias
// correction counts the steps taken (its factors are kept in the loss-scale
// state, updated by k_scale_update).
__global__ void __launch_bounds__(256) k_adam_scaled(float* __restrict__ p, float* __restrict__ g, float* __restrict__ m,
                                                     float* __restrict__ v, size_t n, size_t mlp_begin, size_t mlp_end,
                                                     size_t unscale_end, float lr_grid, float lr_mlp,
                                                     const NifLossScale* __restrict__ ls) {
    const size_t stride = (size_t)gridDim.x * blockDim.x;
    if (ls->overflow) {
        for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) g[i] = 0.f;
        return;
    }
    const float c1 = ls->c1, c2 = ls->c2;
    const float inv = 1.0f / ls->scale;
    // loads first and the gradient cleared last, as in k_adam (clearing it
    // right after its load serialises each iteration's memory accesses: 7x);
    // four parameters per iteration through 16-byte accesses, then the tail
    const size_t tid = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    const size_t n4 = n / 4;
    auto lr = [&](size_t k) { return (k >= mlp_begin && k < mlp_end) ? lr_mlp : lr_grid; };
    auto unscaled = [&](float gi, size_t k) { return k < unscale_end ? gi * inv : gi; };
    for (size_t j = tid; j < n4; j += stride) {
        const float4 g4 = reinterpret_cast<const float4*>(g)[j];
        float4 p4 = reinterpret_cast<float4*>(p)[j];
        float4 m4 = reinterpret_cast<float4*>(m)[j];
        float4 v4 = reinterpret_cast<float4*>(v)[j];
        const size_t i = 4 * j;
        adam_elem(p4.x, unscaled(g4.x, i), m4.x, v4.x, lr(i), c1, c2);
        adam_elem(p4.y, unscaled(g4.y, i + 1), m4.y, v4.y, lr(i + 1), c1, c2);
        adam_elem(p4.z, unscaled(g4.z, i + 2), m4.z, v4.z, lr(i + 2), c1, c2);
        adam_elem(p4.w, unscaled(g4.w, i + 3), m4.w, v4.w, lr(i + 3), c1, c2);
        reinterpret_cast<float4*>(m)[j] = m4;
        reinterpret_cast<float4*>(v)[j] = v4;
        reinterpret_cast<float4*>(p)[j] = p4;
        reinterpret_cast<float4*>(g)[j] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
    for (size_t i = 4 * n4 + tid; i < n; i += stride) {
        adam_elem(p[i], unscaled(g[i], i), m[i], v[i], lr(i), c1, c2);
        g[i] = 0.f;
    }
}

__global__ void k_scale_update(NifLossScale* ls, int dynamic) {
    if (!ls->overflow) {
        ls->b1t *= 0.9;
        ls->b2t *= 0.99;
        ls->c1 = (float)(1.0 / (1.0 - ls->b1t * 0.9));
        ls->c2 = (float)(1.0 / (1.0 - ls->b2t * 0.99));
    }
    if (ls->overflow) {
        ls->overflow = 0;
        ls->skipped++;
        ls->clean = 0;
        if (dynamic) ls->scale = fmaxf(ls->scale * kScaleBackoff, kScaleMin);
    } else if (++ls->clean >= kScaleInterval) {
        ls->clean = 0;
        if (dynamic) ls->scale = fminf(ls->scale * kScaleGrowth, kScaleMax);
    }
}

// ---------------------------------------------------------------------------
// Frame-loop helpers: shadow rays from primary hits, rescaling of a gradient
// computed on the loss-scaled path.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_shadow_rays(const nif_ray* __restrict__ rays, const nif_hit* __restrict__ hits,
                                                     int n, float lx, float ly, float lz, float eps, float tmax,
                                                     nif_ray* __restrict__ out) {
    int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n) return;
    const nif_ray ray = rays[r];
    const nif_hit hit = hits[r];
    nif_ray o;
    o.d[0] = lx; o.d[1] = ly; o.d[2] = lz;
    if (hit.hit) {
        o.o[0] = ray.o[0] + hit.D * ray.d[0];
        o.o[1] = ray.o[1] + hit.D * ray.d[1];
        o.o[2] = ray.o[2] + hit.D * ray.d[2];
        o.tmin = eps;
        o.tmax = tmax;
    } else {           // nothing to shade: an empty interval
        o.o[0] = ray.o[0]; o.o[1] = ray.o[1]; o.o[2] = ray.o[2];
        o.tmin = 0.f;
        o.tmax = 0.f;
    }
    out[r] = o;
}

__global__ void k_unscale(float* __restrict__ v, int n, const NifLossScale* __restrict__ ls) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) v[i] /= ls->scale;
}

// ---------------------------------------------------------------------------
// Reconstruction along the segmented ray (Sec. 2.2)
// ---------------------------------------------------------------------------
__device__ __forceinline__ int find_inst_r(const int* inst_off, int n_inst, int r) {
    if (!inst_off || n_inst <= 1) return 0;
    int lo = 0, hi = n_inst - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (__ldg(inst_off + mid) <= r) lo = mid; else hi = mid - 1;
    }
    return lo;
}

__global__ void __launch_bounds__(128) k_reconstruct(const nif_ray* __restrict__ rays, const int* __restrict__ inst_off,
                                                     int n_inst, int n_rays, const float4* __restrict__ poses,
                                                     FieldView f, const uint32_t* __restrict__ offsets,
                                                     const nif_segment* __restrict__ segs,
                                                     const nif_linseg* __restrict__ lin,
                                                     const float* __restrict__ out, int64_t seg_cap,
                                                     const uint32_t* __restrict__ n_valid, int N, int M,
                                                     unsigned cfg_flags, nif_hit* __restrict__ hits, unsigned flags) {
    int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n_rays) return;
    int64_t a = offsets[r], b = offsets[r + 1];
    if (b > seg_cap) b = seg_cap;
    // a ray whose segments lie past the processed count (a query whose
    // segments exceeded its capacity) is reported without a hit
    if (n_valid && b > (int64_t)*n_valid) b = a;
    nif_hit hit;
    hit.D = __int_as_float(0x7f800000);
    hit.n[0] = hit.n[1] = hit.n[2] = 0.f;
    hit.albedo[0] = hit.albedo[1] = hit.albedo[2] = 0.f;
    hit.hit = 0;
    hit.material = 0;
    hit.pad[0] = hit.pad[1] = 0;
    for (int64_t s = a; s < b; s++) {
        const float* z = out + s * NIF_OUT;
        if (!(z[0] > 0.f)) continue;       // sigmoid(occupancy) > 0.5
        hit.hit = 1;
        if (flags & NIF_SHADOW_ONLY) break;
        const float4* R = reinterpret_cast<const float4*>(rays + r);
        float4 r0 = R[0], r1 = R[1];
        float dn = sqrtf(r0.w * r0.w + r1.x * r1.x + r1.y * r1.y);
        nif_linseg L = lin[s];
        float dvox = (cfg_flags & NIF_FLAG_SIGMOID_DISTANCE) ? 1.7320508075688772f * sigmoidf_(z[1]) : fmaxf(z[1], 0.f);
        float trest = dvox / (float)N;
        float tk = L.l_rest > 0.f ? trest * L.l_def / L.l_rest : 0.f;
        tk = fminf(fmaxf(tk, 0.f), L.l_def);
        // collinear entry/exit points: sum_{j<k} (delta_j + l_j) + delta_k = t0(k) |d|
        hit.D = segs[s].t0 * dn + tk;
        float frac = L.l_rest > 0.f ? trest / L.l_rest : 0.f;
        float3 ph = make_float3(L.p0[0] + frac * (L.p1[0] - L.p0[0]), L.p0[1] + frac * (L.p1[1] - L.p0[1]),
                                L.p0[2] + frac * (L.p1[2] - L.p0[2]));
        int inst = find_inst_r(inst_off, n_inst, r);
        float3 nr = make_float3(z[2], z[3], z[4]);
        if (f.d && inst < f.n) {
            // learned field: J_D = J_pose(q) (I + du/dp), q = ph + u(ph), so
            // J_D^-T n = J_pose(q)^-T (I + du/dp)^-T n
            float3 g[3];
            const float3 u = nif_field_eval(f, inst, ph, g);
            nr = nif_solve3_t(make_float3(1.f + g[0].x, g[0].y, g[0].z), make_float3(g[1].x, 1.f + g[1].y, g[1].z),
                              make_float3(g[2].x, g[2].y, 1.f + g[2].z), nr);
            ph = make_float3(ph.x + u.x, ph.y + u.y, ph.z + u.z);
        }
        float3 j0, j1, j2;
        nif_jacobian_cols(ph, poses[inst], j0, j1, j2);
        // J^-T n is proportional to n.x (j1 x j2) + n.y (j2 x j0) + n.z (j0 x j1), det J > 0
        float3 c0 = nif_cross(j1, j2), c1 = nif_cross(j2, j0), c2 = nif_cross(j0, j1);
        float nx = nr.x * c0.x + nr.y * c1.x + nr.z * c2.x;
        float ny = nr.x * c0.y + nr.y * c1.y + nr.z * c2.y;
        float nz = nr.x * c0.z + nr.y * c1.z + nr.z * c2.z;
        float nl = sqrtf(nx * nx + ny * ny + nz * nz);
        float il = nl > 1e-30f ? 1.0f / nl : 0.f;
        hit.n[0] = nx * il; hit.n[1] = ny * il; hit.n[2] = nz * il;
#pragma unroll
        for (int c = 0; c < 3; c++) hit.albedo[c] = sigmoidf_(z[5 + c]);
        int best = 0;
        for (int c = 1; c < M; c++)
            if (z[8 + c] > z[8 + best]) best = c;
        hit.material = (unsigned char)best;
        break;
    }
    hits[r] = hit;
}

// ---------------------------------------------------------------------------
// Sampler: splitmix64 stream outputs as uniforms (top 24 bits)
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint64_t mix64(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}
__device__ __forceinline__ float uni(uint64_t seed, uint64_t counter) {
    uint64_t z = mix64(seed + (counter + 1ull) * 0x9E3779B97F4A7C15ull);
    return (float)(z >> 40) * (1.0f / 16777216.0f);
}

// rays[j * n + i] is index i of stream stream0 + j, for j < n_streams
__global__ void k_sample_rays(uint64_t seed, int stream0, int n, int n_streams, nif_ray* __restrict__ rays) {
    int64_t gid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (gid >= (int64_t)n * n_streams) return;
    const int j = (int)(gid / n), i = (int)(gid - (int64_t)j * n);
    const int stream_id = stream0 + j;
    uint64_t base = (((uint64_t)(uint32_t)stream_id << 32) + (uint64_t)i) * 8ull;
    float u0 = uni(seed, base), u1 = uni(seed, base + 1), u2 = uni(seed, base + 2), u3 = uni(seed, base + 3),
          u4 = uni(seed, base + 4);
    float z = 2.0f * u0 - 1.0f;
    float a = 6.2831853071795865f * u1;
    float s = sqrtf(fmaxf(0.f, 1.0f - z * z));
    float sa, ca;
    sincosf(a, &sa, &ca);
    float ox = 0.5f + 2.0f * s * ca, oy = 0.5f + 2.0f * s * sa, oz = 0.5f + 2.0f * z;
    float dx = u2 - ox, dy = u3 - oy, dz = u4 - oz;
    float il = rsqrtf(dx * dx + dy * dy + dz * dz);
    nif_ray r;
    r.o[0] = ox; r.o[1] = oy; r.o[2] = oz;
    r.d[0] = dx * il; r.d[1] = dy * il; r.d[2] = dz * il;
    r.tmin = 0.f;
    r.tmax = 1e30f;
    rays[gid] = r;
}

__global__ void k_count_hits(const nif_label* __restrict__ labels, int64_t n, int* __restrict__ n_hit) {
    int c = 0;
    for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < n; s += (int64_t)gridDim.x * blockDim.x)
        c += labels[s].occ ? 1 : 0;
    for (int o = 16; o > 0; o >>= 1) c += __shfl_down_sync(0xffffffffu, c, o);
    if ((threadIdx.x & 31) == 0 && c) atomicAdd(n_hit, c);
}

}  // namespace

nif_status nif_labels_count_hits(nif_handle* h, const nif_label* labels, int64_t n, cudaStream_t s) {
    NIF_CK(h, cudaMemsetAsync(h->d_count, 0, sizeof(int), s));
    if (n > 0) {
        unsigned g = nif_blocks(n, 256);
        unsigned cap = (unsigned)h->num_sms * 4;
        if (g > cap) g = cap;
        k_count_hits<<<g, 256, 0, s>>>(labels, n, h->d_count);
        NIF_CK_LAUNCH(h);
    }
    return NIF_OK;
}

nif_status nif_labels_run(nif_handle* h, const nif_segment* segs, const nif_linseg* lin, const uint32_t* n_dev,
                          int64_t n_max, nif_label* labels, cudaStream_t s, int* n_hit) {
    NifProf prof_(h, "labels", s);
    if (!n_hit) n_hit = h->d_count;
    if (n_max <= 0) return NIF_OK;
    NIF_CK(h, cudaMemsetAsync(n_hit, 0, sizeof(int), s));
    unsigned g = nif_blocks(n_max, 256);
    unsigned cap = (unsigned)h->num_sms * 8;
    if (g > cap) g = cap;
    k_labels<<<g, 256, 0, s>>>(segs, lin, n_dev, n_max, h->d_tri_ptr, h->d_tri_idx, h->d_tri_geo, h->d_alb,
                               h->d_mat, labels, n_hit, (uint32_t)((int64_t)h->N * h->N * h->N), h->n_tris);
    NIF_CK_LAUNCH(h);
    return NIF_OK;
}

nif_status nif_tri_geo_run(nif_handle* h, cudaStream_t s) {
    if (h->n_tris <= 0) return NIF_OK;
    k_tri_geo<<<nif_blocks(h->n_tris, 256), 256, 0, s>>>(h->d_verts, h->d_tris, h->n_tris, h->d_tri_geo);
    NIF_CK_LAUNCH(h);
    return NIF_OK;
}

nif_status nif_loss_run(nif_handle* h, const float* out, const nif_label* labels, const nif_linseg* lin,
                        const uint32_t* n_dev, int64_t n_max, float* dout, cudaStream_t s, bool want_ds,
                        const int* n_hit) {
    NifProf prof_(h, "loss", s);
    if (!n_hit) n_hit = h->d_count;
    NIF_CK(h, cudaMemsetAsync(h->d_lossacc, 0, sizeof(double) * 16, s));
    double* parts = nullptr;
    unsigned g = 0;
    if (n_max > 0) {
        g = nif_blocks(n_max, 256);
        unsigned cap = (unsigned)h->num_sms * 8;
        if (g > cap) g = cap;
        if (h->det) {
            nif_status st = nif_grow(h, h->b_lparts, sizeof(double) * 5 * (size_t)g);
            if (st != NIF_OK) return st;
            parts = (double*)h->b_lparts.p;
        }
        k_loss<<<g, 256, 0, s>>>(out, labels, lin, n_dev, n_max, n_hit, h->d_params + h->off_s, h->N,
                                 h->cfg.n_materials, h->cfg.flags, dout, h->d_lossacc, parts);
        NIF_CK_LAUNCH(h);
    }
    k_loss_final<<<1, 32, 0, s>>>(h->d_lossacc, parts, (int)g, n_dev, n_max, n_hit, h->d_params + h->off_s,
                                  h->cfg.flags, want_ds ? h->d_grad + h->off_s : nullptr, h->d_status);
    NIF_CK_LAUNCH(h);
    return NIF_OK;
}

// grad[e] += part[0][e] + part[1][e] + ... in row-range order (deterministic
// mode's weight gradients: each range's sum was stored, not added in L2)
__global__ void __launch_bounds__(256) k_sum_parts(const float* __restrict__ part, int ny, int64_t cnt,
                                                   float* __restrict__ grad) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < cnt; e += (int64_t)gridDim.x * blockDim.x) {
        float t = 0.f;
        for (int y = 0; y < ny; y++) t += part[(int64_t)y * cnt + e];
        grad[e] += t;
    }
}

nif_status nif_sum_parts_run(nif_handle* h, const float* part, int ny, int64_t cnt, float* grad, cudaStream_t s) {
    if (cnt <= 0 || ny <= 0) return NIF_OK;
    const unsigned g = (unsigned)std::min<int64_t>(nif_blocks(cnt, 256), (int64_t)h->num_sms * 8);
    k_sum_parts<<<g, 256, 0, s>>>(part, ny, cnt, grad);
    NIF_CK_LAUNCH(h);
    return NIF_OK;
}

nif_status nif_adam_split_run(nif_handle* h, float lr_grid, float lr_mlp, cudaStream_t s_tab, cudaStream_t s_w,
                              bool* split) {
    const size_t cut = h->off_layer[0];          // tables [0, cut), weights and log-variances [cut, n_params)
    *split = cut % 4 == 0 && h->off_tables == 0 && cut < h->n_params;
    if (!*split) return NIF_OK;
    h->adam_step++;
    const double c1 = 1.0 / (1.0 - pow(0.9, (double)h->adam_step));
    const double c2 = 1.0 / (1.0 - pow(0.99, (double)h->adam_step));
    const unsigned cap = (unsigned)h->num_sms * 16;
    {
        NifProf prof_(h, "adam", s_tab);
        unsigned g = std::min(nif_blocks((int64_t)cut, 256), cap);
        // relative to the range: no element of [0, cut) lies in [cut, off_s)
        k_adam<<<g, 256, 0, s_tab>>>(h->d_params, h->d_grad, h->d_m, h->d_v, cut, cut, cut, lr_grid, lr_mlp,
                                      (float)c1, (float)c2);
        NIF_CK_LAUNCH(h);
    }
    {
        NifProf prof_(h, "adam_weights", s_w);
        const size_t n = h->n_params - cut;
        unsigned g = std::min(nif_blocks((int64_t)n, 256), cap);
        k_adam<<<g, 256, 0, s_w>>>(h->d_params + cut, h->d_grad + cut, h->d_m + cut, h->d_v + cut, n, 0,
                                    h->off_s - cut, lr_grid, lr_mlp, (float)c1, (float)c2);
        NIF_CK_LAUNCH(h);
    }
    h->lowp_dirty = true;
    h->x3_dirty = true;
    return NIF_OK;
}

nif_status nif_adam_run(nif_handle* h, float lr_grid, float lr_mlp, cudaStream_t s) {
    NifProf prof_(h, "adam", s);
    h->adam_step++;
    double c1 = 1.0 / (1.0 - pow(0.9, (double)h->adam_step));
    double c2 = 1.0 / (1.0 - pow(0.99, (double)h->adam_step));
    unsigned g = nif_blocks((int64_t)h->n_params, 256);
    unsigned cap = (unsigned)h->num_sms * 16;
    if (g > cap) g = cap;
    k_adam<<<g, 256, 0, s>>>(h->d_params, h->d_grad, h->d_m, h->d_v, h->n_params, h->off_layer[0], h->off_s,
                             lr_grid, lr_mlp, (float)c1, (float)c2);
    NIF_CK_LAUNCH(h);
    h->lowp_dirty = true;
    h->x3_dirty = true;
    return NIF_OK;
}

nif_status nif_shadow_rays_run(nif_handle* h, const nif_ray* rays, const nif_hit* hits, int n, const float* light,
                               float eps, float tmax, nif_ray* out, cudaStream_t s) {
    NifProf prof_(h, "shadow_rays", s);
    if (n <= 0) return NIF_OK;
    k_shadow_rays<<<nif_blocks(n, 256), 256, 0, s>>>(rays, hits, n, light[0], light[1], light[2], eps, tmax, out);
    NIF_CK_LAUNCH(h);
    return NIF_OK;
}

nif_status nif_unscale_run(nif_handle* h, float* v, int n, cudaStream_t s) {
    if (n <= 0) return NIF_OK;
    k_unscale<<<nif_blocks(n, 256), 256, 0, s>>>(v, n, h->d_ls);
    NIF_CK_LAUNCH(h);
    return NIF_OK;
}

nif_status nif_grad_check_run(nif_handle* h, cudaStream_t s) {
    NifProf prof_(h, "grad_check", s);
    unsigned g = nif_blocks((int64_t)(h->off_s / 4 + 1), 256);
    unsigned cap = (unsigned)h->num_sms * 8;
    if (g > cap) g = cap;
    k_grad_check<<<g, 256, 0, s>>>(h->d_grad, h->off_s, h->d_ls);
    NIF_CK_LAUNCH(h);
    return NIF_OK;
}

nif_status nif_adam_scaled_run(nif_handle* h, float lr_grid, float lr_mlp, cudaStream_t s) {
    NifProf prof_(h, "adam", s);
    h->adam_step++;
    unsigned g = nif_blocks((int64_t)h->n_params, 256);
    unsigned cap = (unsigned)h->num_sms * 16;
    if (g > cap) g = cap;
    k_adam_scaled<<<g, 256, 0, s>>>(h->d_params, h->d_grad, h->d_m, h->d_v, h->n_params, h->off_layer[0], h->off_s,
                                    h->off_s, lr_grid, lr_mlp, h->d_ls);
    NIF_CK_LAUNCH(h);
    k_scale_update<<<1, 1, 0, s>>>(h->d_ls, h->cfg.precision == NIF_FP16 ? 1 : 0);
    NIF_CK_LAUNCH(h);
    h->lowp_dirty = true;
    h->x3_dirty = true;
    return NIF_OK;
}

nif_status nif_reconstruct_run(nif_handle* h, const nif_ray* rays, const int* inst_off, int n_inst, int n_rays,
                               const uint32_t* offsets, const nif_segment* segs, int64_t seg_cap,
                               const nif_linseg* lin, const float* out, nif_hit* hits, unsigned flags,
                               cudaStream_t s, const uint32_t* n_valid) {
    NifProf prof_(h, "reconstruct", s);
    if (n_rays <= 0) return NIF_OK;
    k_reconstruct<<<nif_blocks(n_rays, 128), 128, 0, s>>>(rays, inst_off, n_inst, n_rays, h->d_pose,
                                                          nif_field_view(h), offsets, segs,
                                                          lin, out, seg_cap, n_valid, h->N, h->cfg.n_materials,
                                                          h->cfg.flags,
                                                          hits, flags);
    NIF_CK_LAUNCH(h);
    return NIF_OK;
}

nif_status nif_sample_rays_run(nif_handle* h, unsigned long long seed, int stream_id, int n, nif_ray* rays,
                               cudaStream_t s, int n_streams) {
    NifProf prof_(h, "sample_rays", s);
    if (n <= 0 || n_streams <= 0) return NIF_OK;
    k_sample_rays<<<nif_blocks((int64_t)n * n_streams, 256), 256, 0, s>>>(seed, stream_id, n, n_streams, rays);
    NIF_CK_LAUNCH(h);
    return NIF_OK;
}
