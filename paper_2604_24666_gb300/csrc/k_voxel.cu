// k_voxel.cu -- rest-space voxelization of the mesh (Sec. 2) and the list of
// triangles overlapping each voxel (used by the ground-truth labels).
//
// Overlap test: separating-axis theorem for a triangle against an axis-aligned
// box (Akenine-Moeller, "Fast 3D triangle-box overlap testing", 2001), voxel
// boxes dilated by 1e-7, in IEEE double with every product and sum explicitly
// rounded (no fused multiply-add), so that the integer occupancy is a fixed
// function of the float32 mesh: the same decision as any other IEEE-double
// evaluation of the same formula in the same order.
#include "nif_internal.cuh"

namespace {

constexpr double kEpsV = 1e-7;

__device__ __forceinline__ double dmul(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ double dadd(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ double dsub(double a, double b) { return __dsub_rn(a, b); }

__device__ bool plane_box(const double n[3], const double v[3], double h) {
    double vmin[3], vmax[3];
    for (int q = 0; q < 3; q++) {
        if (n[q] > 0.0) { vmin[q] = dsub(-h, v[q]); vmax[q] = dsub(h, v[q]); }
        else            { vmin[q] = dsub(h, v[q]);  vmax[q] = dsub(-h, v[q]); }
    }
    double dmin = dadd(dadd(dmul(n[0], vmin[0]), dmul(n[1], vmin[1])), dmul(n[2], vmin[2]));
    double dmax = dadd(dadd(dmul(n[0], vmax[0]), dmul(n[1], vmax[1])), dmul(n[2], vmax[2]));
    if (dmin > 0.0) return false;
    return dmax >= 0.0;
}

__device__ bool tri_box(const double c[3], double h, const double* a, const double* b, const double* d) {
    double v[3][3], e[3][3];
    for (int q = 0; q < 3; q++) {
        v[0][q] = dsub(a[q], c[q]);
        v[1][q] = dsub(b[q], c[q]);
        v[2][q] = dsub(d[q], c[q]);
    }
    for (int q = 0; q < 3; q++) {
        e[0][q] = dsub(v[1][q], v[0][q]);
        e[1][q] = dsub(v[2][q], v[1][q]);
        e[2][q] = dsub(v[0][q], v[2][q]);
    }
    // nine axes e_i x unit_ax
    for (int i = 0; i < 3; i++) {
        for (int ax = 0; ax < 3; ax++) {
            int u = ax == 2 ? 0 : ax + 1;
            int w = ax == 0 ? 2 : ax - 1;
            double p0 = dsub(dmul(e[i][w], v[0][u]), dmul(e[i][u], v[0][w]));
            double p1 = dsub(dmul(e[i][w], v[1][u]), dmul(e[i][u], v[1][w]));
            double p2 = dsub(dmul(e[i][w], v[2][u]), dmul(e[i][u], v[2][w]));
            double rad = dmul(dadd(fabs(e[i][w]), fabs(e[i][u])), h);
            double mn = p0, mx = p0;
            if (p1 < mn) mn = p1;
            if (p1 > mx) mx = p1;
            if (p2 < mn) mn = p2;
            if (p2 > mx) mx = p2;
            if (mn > rad || mx < -rad) return false;
        }
    }
    // three box normals
    for (int q = 0; q < 3; q++) {
        double mn = v[0][q], mx = v[0][q];
        if (v[1][q] < mn) mn = v[1][q];
        if (v[1][q] > mx) mx = v[1][q];
        if (v[2][q] < mn) mn = v[2][q];
        if (v[2][q] > mx) mx = v[2][q];
        if (mn > h || mx < -h) return false;
    }
    double n[3] = {dsub(dmul(e[0][1], e[1][2]), dmul(e[0][2], e[1][1])),
                   dsub(dmul(e[0][2], e[1][0]), dmul(e[0][0], e[1][2])),
                   dsub(dmul(e[0][0], e[1][1]), dmul(e[0][1], e[1][0]))};
    return plane_box(n, v[0], h);
}

// pass 0: occupancy + per-voxel counts; pass 1: fill the lists
__global__ void k_vox_pairs(const float* __restrict__ verts, const int* __restrict__ tris, int nt, int N,
                            uint8_t* __restrict__ occ, uint32_t* __restrict__ cnt,
                            const uint32_t* __restrict__ ptr, int32_t* __restrict__ idx, int pass) {
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nt) return;
    double P[3][3];
    double lo[3] = {1e30, 1e30, 1e30}, hi[3] = {-1e30, -1e30, -1e30};
    for (int k = 0; k < 3; k++) {
        int vi = tris[3 * t + k];
        for (int q = 0; q < 3; q++) {
            P[k][q] = (double)verts[3 * vi + q];
            lo[q] = fmin(lo[q], P[k][q]);
            hi[q] = fmax(hi[q], P[k][q]);
        }
    }
    int i0[3], i1[3];
    for (int q = 0; q < 3; q++) {
        i0[q] = (int)floor((lo[q] - 2 * kEpsV) * N) - 1;
        i1[q] = (int)floor((hi[q] + 2 * kEpsV) * N) + 1;
        i0[q] = max(i0[q], 0);
        i1[q] = min(i1[q], N - 1);
    }
    double h = __dadd_rn(__ddiv_rn(0.5, (double)N), kEpsV);
    for (int k = i0[2]; k <= i1[2]; k++)
        for (int j = i0[1]; j <= i1[1]; j++)
            for (int i = i0[0]; i <= i1[0]; i++) {
                double c[3] = {__ddiv_rn((double)i + 0.5, (double)N), __ddiv_rn((double)j + 0.5, (double)N),
                               __ddiv_rn((double)k + 0.5, (double)N)};
                if (!tri_box(c, h, P[0], P[1], P[2])) continue;
                int64_t v = i + (int64_t)N * (j + (int64_t)N * k);
                if (pass == 0) {
                    occ[v] = 1;
                    atomicAdd(cnt + v, 1u);
                } else {
                    uint32_t pos = ptr[v] + atomicAdd(cnt + v, 1u);
                    idx[pos] = t;
                }
            }
}

// ascending triangle ids within each voxel's list
__global__ void k_sort_lists(const uint32_t* __restrict__ ptr, int32_t* __restrict__ idx, int64_t nvox) {
    int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= nvox) return;
    uint32_t a = ptr[v], b = ptr[v + 1];
    for (uint32_t x = a + 1; x < b; x++) {
        int32_t key = idx[x];
        uint32_t y = x;
        while (y > a && idx[y - 1] > key) {
            idx[y] = idx[y - 1];
            y--;
        }
        idx[y] = key;
    }
}

}  // namespace

nif_status nif_voxelize_run(nif_handle* h) {
    int N = h->N;
    int64_t nvox = (int64_t)N * N * N;
    uint32_t* cnt = nullptr;
    NIF_CK(h, cudaMalloc(&h->d_occ, nvox));
    NIF_CK(h, cudaMalloc(&h->d_tri_ptr, sizeof(uint32_t) * (nvox + 1)));
    NIF_CK(h, cudaMalloc(&cnt, sizeof(uint32_t) * nvox));
    NIF_CK(h, cudaMemset(h->d_occ, 0, nvox));
    NIF_CK(h, cudaMemset(cnt, 0, sizeof(uint32_t) * nvox));
    unsigned g = nif_blocks(h->n_tris, 128);
    if (h->n_tris > 0) {
        k_vox_pairs<<<g, 128>>>(h->d_verts, h->d_tris, h->n_tris, N, h->d_occ, cnt, nullptr, nullptr, 0);
        NIF_CK_LAUNCH(h);
    }
    if (nvox > 0x7fffffff) { cudaFree(cnt); return nif_fail(h, NIF_ERR_ARG, "voxel grid too large"); }
    nif_status st = nif_scan_run(h, cnt, h->d_tri_ptr, (int)nvox, 0);
    if (st != NIF_OK) { cudaFree(cnt); return st; }
    uint32_t total = 0;
    NIF_CK(h, cudaMemcpy(&total, h->d_tri_ptr + nvox, sizeof(uint32_t), cudaMemcpyDeviceToHost));
    h->n_pairs = total;
    NIF_CK(h, cudaMalloc(&h->d_tri_idx, sizeof(int32_t) * (total ? total : 1)));
    NIF_CK(h, cudaMemset(cnt, 0, sizeof(uint32_t) * nvox));
    if (h->n_tris > 0) {
        k_vox_pairs<<<g, 128>>>(h->d_verts, h->d_tris, h->n_tris, N, h->d_occ, cnt, h->d_tri_ptr, h->d_tri_idx, 1);
        NIF_CK_LAUNCH(h);
    }
    k_sort_lists<<<nif_blocks(nvox, 256), 256>>>(h->d_tri_ptr, h->d_tri_idx, nvox);
    NIF_CK_LAUNCH(h);
    NIF_CK(h, cudaDeviceSynchronize());
    cudaFree(cnt);
    return NIF_OK;
}
