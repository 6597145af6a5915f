// nif_field.cu -- the learned deformation field of a handle's instances
// (the paper names learning deformation fields jointly with intersection
// prediction as future work, Sec. 4; the reading is ours): per instance a
// lattice of G^3 rest-space displacements, trilinear, composed before the
// parameterised deformation, D(p) = D_pose(p + u(p)). Setting, reading, and
// the gradient of a loss with respect to it; the fitting step that updates
// it is nif_field_step (nif_api.cu).
#include <cmath>
#include <cstring>
#include <vector>

#include "nif_internal.cuh"

namespace {

// The Lipschitz bound of one instance's field, as k_field_lipschitz computes
// it on the device: within a cell, du/dp_a is a convex combination of the
// cell's four edge differences along a times (G - 1).
double field_lipschitz_host(const float* d, int G) {
    auto at = [&](int i, int j, int k, int c) { return (double)d[(((int64_t)k * G + j) * G + i) * 3 + c]; };
    auto dist = [&](int i0, int j0, int k0, int i1, int j1, int k1) {
        double s = 0.0;
        for (int c = 0; c < 3; c++) {
            const double e = at(i1, j1, k1, c) - at(i0, j0, k0, c);
            s += e * e;
        }
        return std::sqrt(s);
    };
    double best = 0.0;
    for (int k = 0; k + 1 < G; k++)
        for (int j = 0; j + 1 < G; j++)
            for (int i = 0; i + 1 < G; i++) {
                double ex = 0, ey = 0, ez = 0;
                for (int u = 0; u < 2; u++)
                    for (int w = 0; w < 2; w++) {
                        ex = std::max(ex, dist(i, j + u, k + w, i + 1, j + u, k + w));
                        ey = std::max(ey, dist(i + u, j, k + w, i + u, j + 1, k + w));
                        ez = std::max(ez, dist(i + u, j + w, k, i + u, j + w, k + 1));
                    }
                best = std::max(best, (G - 1) * std::sqrt(ex * ex + ey * ey + ez * ez));
            }
    return best;
}

void free_field(nif_handle* h) {
    for (void* p : {(void*)h->d_field, (void*)h->d_field_m, (void*)h->d_field_v, (void*)h->d_field_g,
                    (void*)h->d_field_lip})
        if (p) cudaFree(p);
    h->d_field = h->d_field_m = h->d_field_v = nullptr;
    h->d_field_g = h->d_field_lip = nullptr;
    h->field_G = h->field_n = 0;
    h->field_step = 0;
}

}  // namespace

void nif_field_free(nif_handle* h) { free_field(h); }

extern "C" nif_status nif_set_field(nif_handle* h, int n_inst, int G, const float* delta_host) {
    if (!h) return NIF_ERR_ARG;
    if (n_inst == 0) {
        if (h->n_plans > 0 && h->field_G > 0)
            return nif_fail(h, NIF_ERR_STATE, "destroy the query plans before adding, resizing or removing the field");
        NIF_CK(h, cudaDeviceSynchronize());
        free_field(h);
        return NIF_OK;
    }
    if (n_inst < 0 || G < 2 || G > NIF_FIELD_MAX_G || !delta_host)
        return nif_fail(h, NIF_ERR_ARG, "field: n_inst >= 0, 2 <= G <= 33 and displacements required");
    const int64_t G3 = (int64_t)G * G * G;
    for (int64_t e = 0; e < G3 * 3 * n_inst; e++)
        if (!std::isfinite(delta_host[e])) return nif_fail(h, NIF_ERR_ARG, "field: non-finite displacement");
    for (int i = 0; i < n_inst; i++) {
        const double l = field_lipschitz_host(delta_host + G3 * 3 * i, G);
        if (!(l <= NIF_FIELD_MAX_LIPSCHITZ))
            return nif_fail(h, NIF_ERR_ARG, "field: Lipschitz bound above 0.9 (the inverse needs a contraction)");
    }
    // a query plan's graph holds the field (or its absence) as captured:
    // while plans exist, only the values of an existing field may change
    const bool same = h->field_G == G && h->field_n == n_inst;
    if (!same && h->n_plans > 0)
        return nif_fail(h, NIF_ERR_STATE, "destroy the query plans before adding, resizing or removing the field");
    NIF_CK(h, cudaDeviceSynchronize());
    if (!same) {
        free_field(h);
        const size_t n4 = sizeof(float4) * (size_t)(G3 * n_inst);
        NIF_CK(h, cudaMalloc(&h->d_field, n4));
        NIF_CK(h, cudaMalloc(&h->d_field_m, n4));
        NIF_CK(h, cudaMalloc(&h->d_field_v, n4));
        NIF_CK(h, cudaMalloc(&h->d_field_g, sizeof(float) * 3 * (size_t)(G3 * n_inst)));
        NIF_CK(h, cudaMalloc(&h->d_field_lip, sizeof(float) * (size_t)n_inst));
        h->field_G = G;
        h->field_n = n_inst;
    }
    std::vector<float4> v((size_t)(G3 * n_inst));
    for (size_t e = 0; e < v.size(); e++)
        v[e] = make_float4(delta_host[3 * e], delta_host[3 * e + 1], delta_host[3 * e + 2], 0.f);
    NIF_CK(h, cudaMemcpy(h->d_field, v.data(), sizeof(float4) * v.size(), cudaMemcpyHostToDevice));
    NIF_CK(h, cudaMemset(h->d_field_m, 0, sizeof(float4) * v.size()));
    NIF_CK(h, cudaMemset(h->d_field_v, 0, sizeof(float4) * v.size()));
    NIF_CK(h, cudaMemset(h->d_field_g, 0, sizeof(float) * 3 * v.size()));
    h->field_step = 0;
    return NIF_OK;
}

extern "C" nif_status nif_get_field(nif_handle* h, int* n_inst_host, int* G_host, float* delta_host, size_t bytes) {
    if (!h) return NIF_ERR_ARG;
    if (n_inst_host) *n_inst_host = h->field_n;
    if (G_host) *G_host = h->field_G;
    if (!delta_host) return NIF_OK;
    const size_t n = (size_t)h->field_G * h->field_G * h->field_G * h->field_n;
    if (bytes != sizeof(float) * 3 * n) return nif_fail(h, NIF_ERR_ARG, "field: size mismatch");
    std::vector<float4> v(n);
    NIF_CK(h, cudaDeviceSynchronize());
    if (n) NIF_CK(h, cudaMemcpy(v.data(), h->d_field, sizeof(float4) * n, cudaMemcpyDeviceToHost));
    for (size_t e = 0; e < n; e++) {
        delta_host[3 * e] = v[e].x;
        delta_host[3 * e + 1] = v[e].y;
        delta_host[3 * e + 2] = v[e].z;
    }
    return NIF_OK;
}

extern "C" nif_status nif_field_gradient(nif_handle* h, const nif_pose* poses, int n_inst, const int* inst_off,
                                         const nif_segment* segs, const nif_linseg* lin, int64_t n,
                                         const float* dfeats, float* dfield, void* stream) {
    if (!h) return NIF_ERR_ARG;
    nif_status st = nif_check_inst(h, poses, n_inst, inst_off, 0);
    if (st != NIF_OK) return st;
    if (h->field_G == 0) return nif_fail(h, NIF_ERR_STATE, "the handle has no field (nif_set_field)");
    if (n < 0 || (n > 0 && (!segs || !lin || !dfeats || !dfield))) return nif_fail(h, NIF_ERR_ARG, "buffers");
    cudaStream_t s = (cudaStream_t)stream;
    if ((st = nif_grow(h, h->b_dx, sizeof(float) * 6 * (size_t)std::max<int64_t>(n, 1))) != NIF_OK) return st;
    float* dp = (float*)h->b_dx.p;
    if ((st = nif_encode_segments_dp_run(h, lin, nullptr, n, dfeats, dp, s)) != NIF_OK) return st;
    return nif_field_grad_run(h, segs, lin, dp, nullptr, n, inst_off, n_inst, dfield, s);
}
