// k_segment.cu -- per-pose refit of the deformed-voxel octree, ray / deformed
// voxel segment generation (Sec. 2.1, Sec. 2.2), exclusive scan, and the local
// linearization of each segment into rest space (Sec. 2).
//
// Segment definition (shared with the header): every occupied voxel whose
// deformed hull is hit at least twice gives [max(t_lo, tmin), min(t_hi, tmax)]
// when non-empty; the hull is the hexahedron of the voxel's 8 deformed lattice
// corners with each face split along the diagonal from its lowest lattice
// corner. Hull hits use the watertight ray/triangle test of Woop, Benthin and
// Wald (JCGT 2013): every edge function is evaluated once per canonical
// (low-id, high-id) corner pair with explicitly rounded FP32 operations, so a
// face shared by two voxels gives bit-identical decisions and hit distances in
// both.
//
// The paper starts the traversal with a BVH over the deformed voxels and then
// walks exit faces; here the per-pose BVH (an octree over the occupied voxels
// in Morton order whose boxes are refitted per pose) enumerates every occupied
// hull the ray can meet, which yields the same segment set by definition and
// needs no walk through empty voxels.
#include <algorithm>

#include "nif_internal.cuh"

namespace {

constexpr float kBoxPad = 4e-6f;   // absolute dilation of refitted boxes

// ---------------------------------------------------------------------------
// Refit
// ---------------------------------------------------------------------------
__global__ void k_refit_leaves(int N, int n_leaves, int n_nodes, int n_inst,
                               const uint32_t* __restrict__ leaf_lat,
                               const float4* __restrict__ poses, FieldView f, float* __restrict__ corners,
                               float4* __restrict__ aabb) {
    int64_t gid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (gid >= (int64_t)n_leaves * n_inst) return;
    int inst = (int)(gid / n_leaves);
    int leaf = (int)(gid - (int64_t)inst * n_leaves);
    uint32_t lat = leaf_lat[leaf];
    int i = lat & 1023, j = (lat >> 10) & 1023, k = (lat >> 20) & 1023;
    float4 pose = poses[inst];
    float invN = 1.0f / (float)N;   // exact: N is a power of two
    float* C = corners + ((int64_t)inst * n_leaves + leaf) * 24;
    float3 lo = make_float3(1e30f, 1e30f, 1e30f), hi = make_float3(-1e30f, -1e30f, -1e30f);
#pragma unroll
    for (int c = 0; c < 8; c++) {
        float3 x = make_float3((float)(i + (c & 1)) * invN, (float)(j + ((c >> 1) & 1)) * invN,
                               (float)(k + ((c >> 2) & 1)) * invN);
        if (f.d && inst < f.n) {          // learned field: D = D_pose(x + u(x))
            const float3 u = nif_field_eval(f, inst, x, nullptr);
            x = make_float3(x.x + u.x, x.y + u.y, x.z + u.z);
        }
        float3 y = nif_deform(x, pose);
        C[3 * c + 0] = y.x;
        C[3 * c + 1] = y.y;
        C[3 * c + 2] = y.z;
        lo = make_float3(fminf(lo.x, y.x), fminf(lo.y, y.y), fminf(lo.z, y.z));
        hi = make_float3(fmaxf(hi.x, y.x), fmaxf(hi.y, y.y), fmaxf(hi.z, y.z));
    }
    float4* B = aabb + ((int64_t)inst * n_nodes + leaf) * 2;
    B[0] = make_float4(lo.x - kBoxPad, lo.y - kBoxPad, lo.z - kBoxPad, 0.f);
    B[1] = make_float4(hi.x + kBoxPad, hi.y + kBoxPad, hi.z + kBoxPad, 0.f);
}

__global__ void k_refit_level(int level_begin, int level_count, int n_leaves, int n_nodes,
                              int n_inst, const int2* __restrict__ child, float4* __restrict__ aabb) {
    int64_t gid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (gid >= (int64_t)level_count * n_inst) return;
    int inst = (int)(gid / level_count);
    int node = level_begin + (int)(gid - (int64_t)inst * level_count);
    int2 ch = child[node - n_leaves];
    float4* A = aabb + (int64_t)inst * n_nodes * 2;
    float4 lo = make_float4(1e30f, 1e30f, 1e30f, 0.f), hi = make_float4(-1e30f, -1e30f, -1e30f, 0.f);
    for (int c = ch.x; c < ch.x + ch.y; c++) {
        float4 a = A[2 * c], b = A[2 * c + 1];
        lo.x = fminf(lo.x, a.x); lo.y = fminf(lo.y, a.y); lo.z = fminf(lo.z, a.z);
        hi.x = fmaxf(hi.x, b.x); hi.y = fmaxf(hi.y, b.y); hi.z = fmaxf(hi.z, b.z);
    }
    A[2 * node] = lo;
    A[2 * node + 1] = hi;
}

// ---------------------------------------------------------------------------
// Traversal
// ---------------------------------------------------------------------------
struct RayPre {
    float ox, oy, oz, dx, dy, dz, tmin, tmax;
    float ix, iy, iz;              // 1/d for the slab test
    int kx, ky, kz;                // Woop's axis permutation
    float Sx, Sy, Sz;              // shear constants
};

__device__ __forceinline__ RayPre ray_pre(const nif_ray* rays, int r) {
    const float4* R = reinterpret_cast<const float4*>(rays + r);
    float4 a = R[0], b = R[1];
    RayPre p;
    p.ox = a.x; p.oy = a.y; p.oz = a.z; p.dx = a.w; p.dy = b.x; p.dz = b.y; p.tmin = b.z; p.tmax = b.w;
    p.ix = 1.0f / p.dx; p.iy = 1.0f / p.dy; p.iz = 1.0f / p.dz;
    float ad[3] = {fabsf(p.dx), fabsf(p.dy), fabsf(p.dz)};
    int kz = ad[0] > ad[1] ? (ad[0] > ad[2] ? 0 : 2) : (ad[1] > ad[2] ? 1 : 2);
    int kx = kz + 1 == 3 ? 0 : kz + 1;
    int ky = kx + 1 == 3 ? 0 : kx + 1;
    float d[3] = {p.dx, p.dy, p.dz};
    if (d[kz] < 0.0f) { int t = kx; kx = ky; ky = t; }
    p.kx = kx; p.ky = ky; p.kz = kz;
    p.Sx = __fdiv_rn(d[kx], d[kz]);
    p.Sy = __fdiv_rn(d[ky], d[kz]);
    p.Sz = __fdiv_rn(1.0f, d[kz]);
    return p;
}

__device__ __forceinline__ bool slab(const RayPre& r, float4 lo, float4 hi) {
    float t0x = (lo.x - r.ox) * r.ix, t1x = (hi.x - r.ox) * r.ix;
    float t0y = (lo.y - r.oy) * r.iy, t1y = (hi.y - r.oy) * r.iy;
    float t0z = (lo.z - r.oz) * r.iz, t1z = (hi.z - r.oz) * r.iz;
    float tn = fmaxf(fmaxf(fminf(t0x, t1x), fminf(t0y, t1y)), fmaxf(fminf(t0z, t1z), r.tmin));
    float tf = fminf(fminf(fmaxf(t0x, t1x), fmaxf(t0y, t1y)), fminf(fmaxf(t0z, t1z), r.tmax));
    return tn <= tf;
}

__device__ __forceinline__ float edge_fn(const float* X, const float* Y, int a, int b) {
    // 2D cross product of the sheared corners a < b (canonical direction)
    return __fsub_rn(__fmul_rn(X[a], Y[b]), __fmul_rn(Y[a], X[b]));
}

// One canonical triangle (A < B < C by lattice order); updates hit count and range.
__device__ __forceinline__ void tri_hit(const float* X, const float* Y, const float* Zs, int A, int B,
                                        int C, int& hits, float& tlo, float& thi) {
    float U = -edge_fn(X, Y, B, C);
    float V = edge_fn(X, Y, A, C);
    float W = -edge_fn(X, Y, A, B);
    bool neg = (U < 0.f) || (V < 0.f) || (W < 0.f);
    bool pos = (U > 0.f) || (V > 0.f) || (W > 0.f);
    if (neg && pos) return;
    float det = __fadd_rn(__fadd_rn(U, V), W);
    if (det == 0.f) return;
    float T = __fadd_rn(__fadd_rn(__fmul_rn(U, Zs[A]), __fmul_rn(V, Zs[B])), __fmul_rn(W, Zs[C]));
    float t = __fdiv_rn(T, det);
    hits++;
    tlo = fminf(tlo, t);
    thi = fmaxf(thi, t);
}

// Hull of one voxel: returns true and [t0, t1] when it forms a segment.
__device__ __forceinline__ bool hull_segment(const RayPre& r, const float* __restrict__ C, float& t0,
                                             float& t1) {
    float X[8], Y[8], Zs[8];
    const float4* C4 = reinterpret_cast<const float4*>(C);
    float c[24];
#pragma unroll
    for (int q = 0; q < 6; q++) {
        float4 v = __ldg(C4 + q);
        c[4 * q] = v.x; c[4 * q + 1] = v.y; c[4 * q + 2] = v.z; c[4 * q + 3] = v.w;
    }
    float o[3] = {r.ox, r.oy, r.oz};
#pragma unroll
    for (int k = 0; k < 8; k++) {
        float A[3] = {__fsub_rn(c[3 * k], o[0]), __fsub_rn(c[3 * k + 1], o[1]), __fsub_rn(c[3 * k + 2], o[2])};
        float ax = r.kx == 0 ? A[0] : (r.kx == 1 ? A[1] : A[2]);
        float ay = r.ky == 0 ? A[0] : (r.ky == 1 ? A[1] : A[2]);
        float az = r.kz == 0 ? A[0] : (r.kz == 1 ? A[1] : A[2]);
        X[k] = __fsub_rn(ax, __fmul_rn(r.Sx, az));
        Y[k] = __fsub_rn(ay, __fmul_rn(r.Sy, az));
        Zs[k] = __fmul_rn(r.Sz, az);
    }
    int hits = 0;
    float tlo = 3.0e38f, thi = -3.0e38f;
    // faces {lo, s1, s2, hi}: triangles (lo, s1, hi), (lo, s2, hi)
    tri_hit(X, Y, Zs, 0, 2, 6, hits, tlo, thi); tri_hit(X, Y, Zs, 0, 4, 6, hits, tlo, thi);  // x = 0
    tri_hit(X, Y, Zs, 1, 3, 7, hits, tlo, thi); tri_hit(X, Y, Zs, 1, 5, 7, hits, tlo, thi);  // x = 1
    tri_hit(X, Y, Zs, 0, 1, 5, hits, tlo, thi); tri_hit(X, Y, Zs, 0, 4, 5, hits, tlo, thi);  // y = 0
    tri_hit(X, Y, Zs, 2, 3, 7, hits, tlo, thi); tri_hit(X, Y, Zs, 2, 6, 7, hits, tlo, thi);  // y = 1
    tri_hit(X, Y, Zs, 0, 1, 3, hits, tlo, thi); tri_hit(X, Y, Zs, 0, 2, 3, hits, tlo, thi);  // z = 0
    tri_hit(X, Y, Zs, 4, 5, 7, hits, tlo, thi); tri_hit(X, Y, Zs, 4, 6, 7, hits, tlo, thi);  // z = 1
    if (hits < 2) return false;
    t0 = fmaxf(tlo, r.tmin);
    t1 = fminf(thi, r.tmax);
    return t1 > t0;
}

// One face as the bilinear patch S(u,v) of its corners (lo, s1, s2, hi) =
// (P00, P10, P01, P11) in the sheared ray frame, where the ray is the z axis
// and Zs at a point of the ray is its t: a hit is a root of X(u,v) = Y(u,v) = 0
// with u, v in [0,1]. With h, e, f, g the 2D terms of S (P00, P10 - P00,
// P01 - P00, P11 - P10 - P01 + P00) and k(a,b) = a_x b_y - a_y b_x, u solves
// k(e,g) u^2 + (k(h,g) + k(e,f)) u + k(h,f) = 0 and v follows from
// h + u e + v (f + u g) = 0; t is the bilinear blend of the corners' Zs.
__device__ __forceinline__ float cross2(float ax, float ay, float bx, float by) {
    return fmaf(ax, by, -ay * bx);
}

__device__ __forceinline__ void patch_hit(const float* X, const float* Y, const float* Zs, int lo, int s1, int s2,
                                          int hi, int& hits, float& tlo, float& thi) {
    const float hx = X[lo], hy = Y[lo];
    const float ex = X[s1] - hx, ey = Y[s1] - hy;
    const float fx = X[s2] - hx, fy = Y[s2] - hy;
    const float gx = (X[hi] - X[s1]) - (X[s2] - hx), gy = (Y[hi] - Y[s1]) - (Y[s2] - hy);
    const float k2 = cross2(ex, ey, gx, gy);
    const float k1 = cross2(hx, hy, gx, gy) + cross2(ex, ey, fx, fy);
    const float k0 = cross2(hx, hy, fx, fy);
    float us[2];
    int nu = 0;
    const float scale = fabsf(k2) + fabsf(k1) + fabsf(k0);
    if (!(scale > 0.f)) return;
    if (fabsf(k2) <= 1e-7f * scale) {
        if (k1 != 0.f) us[nu++] = -k0 / k1;
    } else {
        const float disc = fmaf(k1, k1, -4.f * k2 * k0);
        if (disc < 0.f) return;
        const float sq = sqrtf(disc);
        const float q = -0.5f * (k1 + copysignf(sq, k1));
        us[nu++] = q / k2;
        if (disc > 0.f && q != 0.f) us[nu++] = k0 / q;
    }
    const float zl = Zs[lo], ze = Zs[s1] - zl, zf = Zs[s2] - zl, zg = (Zs[hi] - Zs[s1]) - (Zs[s2] - zl);
#pragma unroll
    for (int i = 0; i < 2; i++) {
        if (i >= nu) break;
        const float u = us[i];
        if (!(u >= 0.f && u <= 1.f)) continue;
        const float wx = fmaf(u, gx, fx), wy = fmaf(u, gy, fy);
        const float rx = fmaf(u, ex, hx), ry = fmaf(u, ey, hy);
        const float ww = fmaf(wx, wx, wy * wy);
        if (!(ww > 0.f)) continue;
        const float v = -fmaf(rx, wx, ry * wy) / ww;
        if (!(v >= 0.f && v <= 1.f)) continue;
        const float t = zl + u * ze + v * fmaf(u, zg, zf);
        hits++;
        tlo = fminf(tlo, t);
        thi = fmaxf(thi, t);
    }
}

// Hull of one voxel with bilinear faces (NIF_FLAG_BILINEAR_FACES): the same
// segment rule as hull_segment, on the six patches.
__device__ __forceinline__ bool hull_segment_bil(const RayPre& r, const float* __restrict__ C, float& t0,
                                                 float& t1) {
    float X[8], Y[8], Zs[8];
    const float4* C4 = reinterpret_cast<const float4*>(C);
    float c[24];
#pragma unroll
    for (int q = 0; q < 6; q++) {
        float4 v = __ldg(C4 + q);
        c[4 * q] = v.x; c[4 * q + 1] = v.y; c[4 * q + 2] = v.z; c[4 * q + 3] = v.w;
    }
    float o[3] = {r.ox, r.oy, r.oz};
#pragma unroll
    for (int k = 0; k < 8; k++) {
        float A[3] = {c[3 * k] - o[0], c[3 * k + 1] - o[1], c[3 * k + 2] - o[2]};
        float ax = r.kx == 0 ? A[0] : (r.kx == 1 ? A[1] : A[2]);
        float ay = r.ky == 0 ? A[0] : (r.ky == 1 ? A[1] : A[2]);
        float az = r.kz == 0 ? A[0] : (r.kz == 1 ? A[1] : A[2]);
        X[k] = fmaf(-r.Sx, az, ax);
        Y[k] = fmaf(-r.Sy, az, ay);
        Zs[k] = r.Sz * az;
    }
    int hits = 0;
    float tlo = 3.0e38f, thi = -3.0e38f;
    patch_hit(X, Y, Zs, 0, 2, 4, 6, hits, tlo, thi);   // x = 0
    patch_hit(X, Y, Zs, 1, 3, 5, 7, hits, tlo, thi);   // x = 1
    patch_hit(X, Y, Zs, 0, 1, 4, 5, hits, tlo, thi);   // y = 0
    patch_hit(X, Y, Zs, 2, 3, 6, 7, hits, tlo, thi);   // y = 1
    patch_hit(X, Y, Zs, 0, 1, 2, 3, hits, tlo, thi);   // z = 0
    patch_hit(X, Y, Zs, 4, 5, 6, 7, hits, tlo, thi);   // z = 1
    if (hits < 2) return false;
    t0 = fmaxf(tlo, r.tmin);
    t1 = fminf(thi, r.tmax);
    return t1 > t0;
}

template <bool BIL>
__device__ __forceinline__ bool hull_test(const RayPre& r, const float* __restrict__ C, float& t0, float& t1) {
    return BIL ? hull_segment_bil(r, C, t0, t1) : hull_segment(r, C, t0, t1);
}

__device__ __forceinline__ int find_inst(const int* inst_off, int n_inst, int r) {
    if (!inst_off || n_inst <= 1) return 0;
    int lo = 0, hi = n_inst - 1;     // largest i with inst_off[i] <= r
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (__ldg(inst_off + mid) <= r) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// Sorting one ray's row of segments by (t0, voxel), in place by insertion
// (rows are short: a few segments per ray).
__device__ __forceinline__ void sort_row_inplace(nif_segment* segs, int64_t base, int64_t end) {
    for (int64_t a = base + 1; a < end; a++) {
        nif_segment key = segs[a];
        int64_t b = a - 1;
        while (b >= base) {
            nif_segment o = segs[b];
            bool gt = o.t0 > key.t0 || (o.t0 == key.t0 && o.voxel > key.voxel);
            if (!gt) break;
            segs[b + 1] = o;
            b--;
        }
        segs[b + 1] = key;
    }
}

constexpr int kStack = 96;

// Modes of the traversal kernel
enum { kModeCount = 0, kModeEmit = 1, kModeTemp = 2 };

// Ray / octree traversal with warp-pooled hull tests. Each thread walks the
// octree of its own ray with a private stack; every leaf whose refitted box
// the ray meets becomes a (lane, leaf) candidate in a per-warp queue in
// shared memory. Whenever 32 candidates are queued (or no lane has work
// left) the warp tests them against their rays' hulls with all 32 lanes at
// once, so the 12-triangle hull test -- the bulk of the arithmetic -- runs
// without divergence.
//   kModeCount: per-ray segment counts;
//   kModeEmit:  segments written to the CSR rows [offsets[r], offsets[r+1])
//               of their ray, then each ray's list sorted by (t0, voxel);
//   kModeTemp:  counts plus every segment appended to `temp` at a
//               warp-reserved position (ray order is restored by a scatter).
template <int MODE, int kTravWarps, bool BIL = false>
__global__ void __launch_bounds__(kTravWarps * 32, 32 / kTravWarps) k_seg_traverse(
    const nif_ray* __restrict__ rays, const int* __restrict__ inst_off, int n_inst, int n_rays,
    TreeView tree, const float* __restrict__ corners, const float4* __restrict__ aabb,
    uint32_t* __restrict__ counts, const uint32_t* __restrict__ offsets, nif_segment* __restrict__ segs,
    int64_t cap, uint32_t* __restrict__ temp_cursor, int64_t emit_skip_le, int* status) {
    // emit as the fallback of a temp pass: nothing to do unless the temp overflowed
    if (MODE == kModeEmit && temp_cursor && (int64_t)*temp_cursor <= emit_skip_le) return;
    __shared__ RayPre s_ray[kTravWarps][32];
    __shared__ uint32_t s_q[kTravWarps][64];
    __shared__ uint32_t s_cnt[kTravWarps][32];
    __shared__ int s_inst[kTravWarps][32];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const unsigned FULL = 0xffffffffu;
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    const int r_warp0 = blockIdx.x * blockDim.x + warp * 32;
    const bool valid = r < n_rays;
    int inst = valid ? find_inst(inst_off, n_inst, r) : 0;
    RayPre ray;
    if (valid) ray = ray_pre(rays, r);
    else ray = RayPre{};
    s_ray[warp][lane] = ray;
    s_cnt[warp][lane] = 0;
    s_inst[warp][lane] = inst;
    const float4* A = aabb + (int64_t)inst * tree.n_nodes * 2;
    // the stack holds nodes whose boxes the ray is known to meet: a node's
    // children are box-tested together when it is expanded (their boxes are
    // contiguous, so the loads go out back to back) and only those hit are
    // pushed; a popped leaf goes straight to the queue
    int stack[kStack];
    int sp = 0;
    if (valid)
        for (int q = tree.top_begin + tree.top_count - 1; q >= tree.top_begin; q--)
            if (slab(ray, __ldg(A + 2 * q), __ldg(A + 2 * q + 1))) stack[sp++] = q;
    __syncwarp();
    int qn = 0;
    while (true) {
        // fill the queue with leaf candidates
        while (qn < 32) {
            bool want = sp > 0;
            if (!__any_sync(FULL, want)) break;
            int cand = -1;
            if (want) {
                int node = stack[--sp];
                if (node < tree.n_leaves) {
                    cand = node;
                } else {
                    int2 ch = __ldg(tree.child + (node - tree.n_leaves));
                    if (sp + ch.y > kStack) {
                        nif_set_status(status, NIF_ERR_CAPACITY);
                        sp = 0;
                    } else {
                        for (int c = ch.x + ch.y - 1; c >= ch.x; c--)
                            if (slab(ray, __ldg(A + 2 * c), __ldg(A + 2 * c + 1))) stack[sp++] = c;
                    }
                }
            }
            unsigned m = __ballot_sync(FULL, cand >= 0);
            if (cand >= 0) s_q[warp][qn + __popc(m & ((1u << lane) - 1u))] = ((uint32_t)lane << 27) | (uint32_t)cand;
            qn += __popc(m);
        }
        __syncwarp();
        if (qn == 0) break;
        const int take = qn < 32 ? qn : 32;
        bool hit = false;
        int L = 0;
        nif_segment sg;
        if (lane < take) {
            uint32_t c = s_q[warp][lane];
            L = (int)(c >> 27);
            int leaf = (int)(c & 0x7FFFFFFu);
            float t0, t1;
            const float* C = corners + ((int64_t)s_inst[warp][L] * tree.n_leaves + leaf) * 24;
            if (hull_test<BIL>(s_ray[warp][L], C, t0, t1)) {
                hit = true;
                sg.ray = (uint32_t)(r_warp0 + L);
                sg.voxel = __ldg(tree.leaf_vox + leaf);
                sg.t0 = t0;
                sg.t1 = t1;
            }
        }
        if (MODE == kModeCount) {
            if (hit) atomicAdd(&s_cnt[warp][L], 1u);
        } else if (MODE == kModeEmit) {
            if (hit) {
                uint32_t pos = atomicAdd(&s_cnt[warp][L], 1u);
                int64_t g = (int64_t)offsets[r_warp0 + L] + pos;
                if (g < (int64_t)offsets[r_warp0 + L + 1] && g < cap) segs[g] = sg;
            }
        } else {
            if (hit) atomicAdd(&s_cnt[warp][L], 1u);
            unsigned hm = __ballot_sync(FULL, hit);
            uint32_t wb = 0;
            if (lane == 0 && hm) wb = atomicAdd(temp_cursor, (uint32_t)__popc(hm));
            wb = __shfl_sync(FULL, wb, 0);
            if (hit) {
                int64_t g = (int64_t)wb + __popc(hm & ((1u << lane) - 1u));
                if (g < cap) segs[g] = sg;
            }
        }
        __syncwarp();
        const int rest = qn - take;
        uint32_t moved = lane < rest ? s_q[warp][32 + lane] : 0u;
        __syncwarp();
        if (lane < rest) s_q[warp][lane] = moved;
        __syncwarp();
        qn = rest;
    }
    __syncwarp();
    if (!valid) return;
    if (MODE != kModeEmit) {
        counts[r] = s_cnt[warp][lane];
        return;
    }
    // sort this ray's segments by (t0, voxel): short runs
    int64_t base = offsets[r], end = offsets[r + 1];
    if (end > cap) end = cap;
    sort_row_inplace(segs, base, end);
}

// ---------------------------------------------------------------------------
// Exit-face walk: the traversal the paper describes (Sec. 2.1). A BVH query
// finds the first occupied hull on the ray; from there the ray walks from
// voxel to voxel through the faces of the deformed hexahedra, empty voxels
// included, emitting the segment of every occupied voxel it enters; when it
// leaves the deformed grid (which is not convex under bending) the BVH is
// queried again for the next occupied hull past the exit. The emitted set is
// the one the enumeration above gives by definition (every segment's t comes
// from the same hull test on the same corners); the walk exists to measure
// the paper's design against the enumeration on this hardware.
// ---------------------------------------------------------------------------
// every lattice point of every instance deformed: [inst][(N+1)^3] (x, y, z, 0),
// computed as k_refit_leaves computes the corners of the occupied voxels
__global__ void k_lattice(int N, int n_inst, const float4* __restrict__ poses, FieldView f, float4* __restrict__ lat) {
    const int M = N + 1;
    const int64_t per = (int64_t)M * M * M;
    const int64_t gid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (gid >= per * n_inst) return;
    const int inst = (int)(gid / per);
    const int64_t p = gid - (int64_t)inst * per;
    const int i = (int)(p % M), j = (int)((p / M) % M), k = (int)(p / ((int64_t)M * M));
    const float invN = 1.0f / (float)N;
    float3 x = make_float3((float)i * invN, (float)j * invN, (float)k * invN);
    if (f.d && inst < f.n) {
        const float3 u = nif_field_eval(f, inst, x, nullptr);
        x = make_float3(x.x + u.x, x.y + u.y, x.z + u.z);
    }
    const float3 y = nif_deform(x, poses[inst]);
    lat[gid] = make_float4(y.x, y.y, y.z, 0.f);
}

// voxel id -> leaf index of the octree (-1: empty)
__global__ void k_vox_leaf(const uint32_t* __restrict__ leaf_vox, int n_leaves, int* __restrict__ map) {
    const int l = blockIdx.x * blockDim.x + threadIdx.x;
    if (l < n_leaves) map[leaf_vox[l]] = l;
}

// Woop et al. on one canonical triangle: true and t when the ray meets it
__device__ __forceinline__ bool tri_t(const float* X, const float* Y, const float* Zs, int A, int B, int C,
                                      float& t) {
    float U = -edge_fn(X, Y, B, C);
    float V = edge_fn(X, Y, A, C);
    float W = -edge_fn(X, Y, A, B);
    bool neg = (U < 0.f) || (V < 0.f) || (W < 0.f);
    bool pos = (U > 0.f) || (V > 0.f) || (W > 0.f);
    if (neg && pos) return false;
    float det = __fadd_rn(__fadd_rn(U, V), W);
    if (det == 0.f) return false;
    float T = __fadd_rn(__fadd_rn(__fmul_rn(U, Zs[A]), __fmul_rn(V, Zs[B])), __fmul_rn(W, Zs[C]));
    t = __fdiv_rn(T, det);
    return true;
}

// Exit of a hull (8 corners c[3*k..] in lattice order): the face other than
// f_in hit at the smallest t >= t_in (t > t_in when f_in < 0); -1 when none.
// Faces 0..5 are x = 0, x = 1, y = 0, y = 1, z = 0, z = 1; their triangles
// are the canonical ones of hull_segment, so the two voxels of a shared face
// take the same decisions.
__device__ __forceinline__ int hull_exit(const RayPre& r, const float* c, int f_in, float t_in, float& t_out) {
    float X[8], Y[8], Zs[8];
    const float o[3] = {r.ox, r.oy, r.oz};
#pragma unroll
    for (int k = 0; k < 8; k++) {
        float A[3] = {__fsub_rn(c[3 * k], o[0]), __fsub_rn(c[3 * k + 1], o[1]), __fsub_rn(c[3 * k + 2], o[2])};
        float ax = r.kx == 0 ? A[0] : (r.kx == 1 ? A[1] : A[2]);
        float ay = r.ky == 0 ? A[0] : (r.ky == 1 ? A[1] : A[2]);
        float az = r.kz == 0 ? A[0] : (r.kz == 1 ? A[1] : A[2]);
        X[k] = __fsub_rn(ax, __fmul_rn(r.Sx, az));
        Y[k] = __fsub_rn(ay, __fmul_rn(r.Sy, az));
        Zs[k] = __fmul_rn(r.Sz, az);
    }
    // triangles (lo, s1, hi), (lo, s2, hi) of each face
    const int tri[6][4] = {{0, 2, 4, 6}, {1, 3, 5, 7}, {0, 1, 4, 5}, {2, 3, 6, 7}, {0, 1, 2, 3}, {4, 5, 6, 7}};
    int best = -1;
    float bt = 3.0e38f;
#pragma unroll
    for (int f = 0; f < 6; f++) {
        if (f == f_in) continue;
        const int lo = tri[f][0], s1 = tri[f][1], s2 = tri[f][2], hi = tri[f][3];
        float tt;
#pragma unroll
        for (int h2 = 0; h2 < 2; h2++) {
            if (tri_t(X, Y, Zs, lo, h2 ? s2 : s1, hi, tt)) {
                const bool ahead = f_in < 0 ? tt > t_in : tt >= t_in;
                if (ahead && tt < bt) { bt = tt; best = f; }
            }
        }
    }
    t_out = bt;
    return best;
}

// slab entry distance of a box, +inf when the ray misses it within [tmin, tmax]
__device__ __forceinline__ float slab_t(const RayPre& r, float4 lo, float4 hi) {
    float t0x = (lo.x - r.ox) * r.ix, t1x = (hi.x - r.ox) * r.ix;
    float t0y = (lo.y - r.oy) * r.iy, t1y = (hi.y - r.oy) * r.iy;
    float t0z = (lo.z - r.oz) * r.iz, t1z = (hi.z - r.oz) * r.iz;
    float tn = fmaxf(fmaxf(fminf(t0x, t1x), fminf(t0y, t1y)), fmaxf(fminf(t0z, t1z), r.tmin));
    float tf = fminf(fminf(fmaxf(t0x, t1x), fmaxf(t0y, t1y)), fminf(fmaxf(t0z, t1z), r.tmax));
    return tn <= tf ? tn : 3.0e38f;
}

// BVH query: the occupied hull whose segment starts first, t0 > t_after
// (t0 >= t_after when incl); ties to the lower voxel id. Boxes that start
// after the best t0 so far are not opened.
__device__ __forceinline__ bool bvh_first(const RayPre& r, const TreeView& tree, const float4* A,
                                          const float* corners, float t_after, bool incl, int& leaf_out,
                                          float& t0_out, float& t1_out, int* status) {
    int stack[kStack];
    int sp = 0;
    for (int q = tree.top_begin + tree.top_count - 1; q >= tree.top_begin; q--)
        if (slab_t(r, __ldg(A + 2 * q), __ldg(A + 2 * q + 1)) < 3.0e38f) stack[sp++] = q;
    float best = 3.0e38f;
    uint32_t best_vox = 0xFFFFFFFFu;
    leaf_out = -1;
    while (sp > 0) {
        const int node = stack[--sp];
        if (node < tree.n_leaves) {
            float t0, t1;
            if (hull_segment(r, corners + (int64_t)node * 24, t0, t1)) {
                const uint32_t vox = __ldg(tree.leaf_vox + node);
                const bool after = incl ? t0 >= t_after : t0 > t_after;
                if (after && (t0 < best || (t0 == best && vox < best_vox))) {
                    best = t0;
                    best_vox = vox;
                    leaf_out = node;
                    t0_out = t0;
                    t1_out = t1;
                }
            }
            continue;
        }
        const int2 ch = __ldg(tree.child + (node - tree.n_leaves));
        if (sp + ch.y > kStack || ch.y > 8) {
            nif_set_status(status, NIF_ERR_CAPACITY);
            return false;
        }
        // children the ray meets before the best start so far, pushed farthest
        // first so that the nearest box is opened next
        float ct[8];
        int cn[8];
        int m = 0;
        for (int c = ch.x; c < ch.x + ch.y; c++) {
            const float tn = slab_t(r, __ldg(A + 2 * c), __ldg(A + 2 * c + 1));
            if (tn < 3.0e38f && tn <= best) {
                int k = m++;
                while (k > 0 && ct[k - 1] < tn) {
                    ct[k] = ct[k - 1];
                    cn[k] = cn[k - 1];
                    k--;
                }
                ct[k] = tn;
                cn[k] = c;
            }
        }
        for (int k = 0; k < m; k++) stack[sp++] = cn[k];
    }
    return leaf_out >= 0;
}

enum { kWalkCount = 0, kWalkEmit = 1, kWalkFirst = 2 };
constexpr int kWalkRecent = 8;   // voxels emitted last, for re-entries of non-convex hulls

// One thread per ray.
//   kWalkCount: per-ray segment counts;
//   kWalkEmit:  segments into the CSR rows [offsets[r], offsets[r+1]), each row
//               then sorted by (t0, voxel);
//   kWalkFirst: 1 where the first BVH query finds a hull (the walk skipped):
//               the BVH part of the traversal alone, for timing.
template <int MODE>
__global__ void __launch_bounds__(128) k_seg_walk(const nif_ray* __restrict__ rays, const int* __restrict__ inst_off,
                                                  int n_inst, int n_rays, int N, TreeView tree,
                                                  const float* __restrict__ corners, const float4* __restrict__ aabb,
                                                  const float4* __restrict__ lat, const int* __restrict__ vox_leaf,
                                                  uint32_t* __restrict__ counts, const uint32_t* __restrict__ offsets,
                                                  nif_segment* __restrict__ segs, int64_t cap, int* status) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n_rays) return;
    const int inst = find_inst(inst_off, n_inst, r);
    const RayPre ray = ray_pre(rays, r);
    const float4* A = aabb + (int64_t)inst * tree.n_nodes * 2;
    const float* C = corners + (int64_t)inst * tree.n_leaves * 24;
    const int M = N + 1;
    const float4* Lt = lat + (int64_t)inst * M * M * M;
    int64_t base = 0, lim = 0;
    if (MODE == kWalkEmit) {
        base = offsets[r];
        lim = (int64_t)offsets[r + 1] < cap ? (int64_t)offsets[r + 1] : cap;
    }
    uint32_t cnt = 0;
    uint32_t recent[kWalkRecent];
    int nrec = 0;
    float t_after = ray.tmin;
    bool incl = true;
    const int max_steps = 4 * N + 16;
    // every query past the first starts beyond the voxels walked so far and
    // finds a new hull, so the number of queries is bounded by the leaves
    for (int q = 0; q <= tree.n_leaves; q++) {
        int leaf;
        float t0, t1;
        if (!bvh_first(ray, tree, A, C, t_after, incl, leaf, t0, t1, status)) break;
        if (MODE == kWalkFirst) { cnt = 1; break; }
        const uint32_t vox0 = __ldg(tree.leaf_vox + leaf);
        int ci = (int)(vox0 % (uint32_t)N), cj = (int)((vox0 / (uint32_t)N) % (uint32_t)N),
            ck = (int)(vox0 / ((uint32_t)N * (uint32_t)N));
        int f_in = -1;
        float t_in = t0, t_exit = t0;
        bool first = true;
        for (int step = 0; step < max_steps; step++) {
            const uint32_t v = (uint32_t)ci + (uint32_t)N * ((uint32_t)cj + (uint32_t)N * (uint32_t)ck);
            const int lf = first ? leaf : __ldg(vox_leaf + v);
            if (lf >= 0) {
                bool seen = false;
                for (int i = 0; i < kWalkRecent && i < nrec; i++) seen |= recent[i] == v;
                float s0 = t0, s1 = t1;
                if (!seen && (first || hull_segment(ray, C + (int64_t)lf * 24, s0, s1))) {
                    if (MODE == kWalkEmit && base + cnt < lim) segs[base + cnt] = nif_segment{(uint32_t)r, v, s0, s1};
                    cnt++;
                    recent[nrec % kWalkRecent] = v;
                    nrec++;
                }
            }
            first = false;
            float c[24];
#pragma unroll
            for (int k = 0; k < 8; k++) {
                const int64_t idx = (int64_t)(ci + (k & 1)) +
                                    (int64_t)M * ((cj + ((k >> 1) & 1)) + (int64_t)M * (ck + ((k >> 2) & 1)));
                const float4 pnt = __ldg(Lt + idx);
                c[3 * k] = pnt.x;
                c[3 * k + 1] = pnt.y;
                c[3 * k + 2] = pnt.z;
            }
            float t_out;
            const int f = hull_exit(ray, c, f_in, t_in, t_out);
            if (f < 0 || t_out > ray.tmax) {   // no exit found (or past tmax): query again past this entry
                t_exit = t_in;
                break;
            }
            ci += f == 0 ? -1 : (f == 1 ? 1 : 0);
            cj += f == 2 ? -1 : (f == 3 ? 1 : 0);
            ck += f == 4 ? -1 : (f == 5 ? 1 : 0);
            t_exit = t_out;
            if (ci < 0 || ci >= N || cj < 0 || cj >= N || ck < 0 || ck >= N) break;   // left the deformed grid
            f_in = f ^ 1;
            t_in = t_out;
        }
        t_after = t_exit;
        incl = false;
    }
    if (MODE != kWalkEmit) {
        counts[r] = cnt;
        return;
    }
    const int64_t end = base + (int64_t)cnt < lim ? base + (int64_t)cnt : lim;
    sort_row_inplace(segs, base, end);
}

// The same traversal with persistent warps that refill idle lanes (count and
// temp modes): rays come from a global counter; a lane whose ray has an empty
// stack and no queued candidates writes its count and takes the next ray, so
// the octree walk keeps most lanes busy instead of waiting for the longest
// ray of a fixed warp (measured 9.9 of 32 lanes active per instruction with
// one ray per thread). Queue entries name a lane, and a lane is refilled only
// once its queued candidates are tested, so an entry always belongs to the
// lane's current ray.
template <int MODE, int kTravWarps, bool BIL = false>
__global__ void __launch_bounds__(kTravWarps * 32, 32 / kTravWarps) k_seg_traverse_p(
    const nif_ray* __restrict__ rays, const int* __restrict__ inst_off, int n_inst, int n_rays,
    TreeView tree, const float* __restrict__ corners, const float4* __restrict__ aabb,
    uint32_t* __restrict__ counts, nif_segment* __restrict__ segs, int64_t cap,
    uint32_t* __restrict__ temp_cursor, uint32_t* __restrict__ ray_next, int* status) {
    static_assert(MODE == kModeCount || MODE == kModeTemp, "count and temp modes");
    __shared__ RayPre s_ray[kTravWarps][32];
    __shared__ uint32_t s_q[kTravWarps][64];
    __shared__ uint32_t s_cnt[kTravWarps][32];
    __shared__ int s_inst[kTravWarps][32];
    __shared__ int s_rid[kTravWarps][32];
    __shared__ int s_pend[kTravWarps][32];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const unsigned FULL = 0xffffffffu;
    int r = -1;                 // this lane's ray, -1 when it has none
    bool exhausted = false;     // warp-uniform: the ray counter ran past n_rays
    int stack[kStack];
    int sp = 0;
    int qn = 0;
    s_pend[warp][lane] = 0;
    __syncwarp();
    while (true) {
        // idle lanes take the next rays, one atomic per warp
        const unsigned im = __ballot_sync(FULL, r < 0 && !exhausted);
        if (im) {
            const int leader = __ffs(im) - 1;
            uint32_t base = 0;
            if (lane == leader) base = atomicAdd(ray_next, (uint32_t)__popc(im));
            base = __shfl_sync(FULL, base, leader);
            if ((im >> lane) & 1u) {
                const uint32_t nr = base + (uint32_t)__popc(im & ((1u << lane) - 1u));
                if (nr < (uint32_t)n_rays) {
                    r = (int)nr;
                    const int inst = find_inst(inst_off, n_inst, r);
                    const RayPre ray = ray_pre(rays, r);
                    s_ray[warp][lane] = ray;
                    s_inst[warp][lane] = inst;
                    s_rid[warp][lane] = r;
                    s_cnt[warp][lane] = 0;
                    const float4* A = aabb + (int64_t)inst * tree.n_nodes * 2;
                    sp = 0;
                    for (int q = tree.top_begin + tree.top_count - 1; q >= tree.top_begin; q--)
                        if (slab(ray, __ldg(A + 2 * q), __ldg(A + 2 * q + 1))) stack[sp++] = q;
                }
            }
            exhausted = (uint64_t)base + (uint64_t)__popc(im) >= (uint64_t)n_rays;
        }
        __syncwarp();
        // fill the queue with leaf candidates
        while (qn < 32) {
            const bool want = sp > 0;
            if (!__any_sync(FULL, want)) break;
            int cand = -1;
            if (want) {
                const int node = stack[--sp];
                if (node < tree.n_leaves) {
                    cand = node;
                } else {
                    // the slab test's 8 ray values in registers for all
                    // children (read from shared memory once per node)
                    const RayPre& rs = s_ray[warp][lane];
                    RayPre ray;
                    ray.ox = rs.ox; ray.oy = rs.oy; ray.oz = rs.oz;
                    ray.ix = rs.ix; ray.iy = rs.iy; ray.iz = rs.iz;
                    ray.tmin = rs.tmin; ray.tmax = rs.tmax;
                    const float4* A = aabb + (int64_t)s_inst[warp][lane] * tree.n_nodes * 2;
                    const int2 ch = __ldg(tree.child + (node - tree.n_leaves));
                    if (sp + ch.y > kStack) {
                        nif_set_status(status, NIF_ERR_CAPACITY);
                        sp = 0;
                    } else {
                        for (int c = ch.x + ch.y - 1; c >= ch.x; c--)
                            if (slab(ray, __ldg(A + 2 * c), __ldg(A + 2 * c + 1))) stack[sp++] = c;
                    }
                }
            }
            const unsigned m = __ballot_sync(FULL, cand >= 0);
            if (cand >= 0) {
                s_q[warp][qn + __popc(m & ((1u << lane) - 1u))] = ((uint32_t)lane << 27) | (uint32_t)cand;
                s_pend[warp][lane]++;
            }
            qn += __popc(m);
        }
        __syncwarp();
        if (qn > 0) {
            // hull tests of up to 32 queued candidates, 32 lanes wide
            const int take = qn < 32 ? qn : 32;
            bool hit = false;
            int L = 0;
            nif_segment sg;
            if (lane < take) {
                const uint32_t c = s_q[warp][lane];
                L = (int)(c >> 27);
                const int leaf = (int)(c & 0x7FFFFFFu);
                float t0, t1;
                const float* C = corners + ((int64_t)s_inst[warp][L] * tree.n_leaves + leaf) * 24;
                if (hull_test<BIL>(s_ray[warp][L], C, t0, t1)) {
                    hit = true;
                    sg.ray = (uint32_t)s_rid[warp][L];
                    sg.voxel = __ldg(tree.leaf_vox + leaf);
                    sg.t0 = t0;
                    sg.t1 = t1;
                }
            }
            if (hit) atomicAdd(&s_cnt[warp][L], 1u);
            if (MODE == kModeTemp) {
                const unsigned hm = __ballot_sync(FULL, hit);
                uint32_t wb = 0;
                if (lane == 0 && hm) wb = atomicAdd(temp_cursor, (uint32_t)__popc(hm));
                wb = __shfl_sync(FULL, wb, 0);
                if (hit) {
                    const int64_t g = (int64_t)wb + __popc(hm & ((1u << lane) - 1u));
                    if (g < cap) segs[g] = sg;
                }
            }
            __syncwarp();
            if (lane < take) atomicSub(&s_pend[warp][L], 1);
            const int rest = qn - take;
            const uint32_t moved = lane < rest ? s_q[warp][32 + lane] : 0u;
            __syncwarp();
            if (lane < rest) s_q[warp][lane] = moved;
            qn = rest;
        }
        __syncwarp();
        // a ray with no stack left and no queued candidates is complete
        if (r >= 0 && sp == 0 && s_pend[warp][lane] == 0) {
            counts[r] = s_cnt[warp][lane];
            r = -1;
        }
        if (exhausted && qn == 0 && !__any_sync(FULL, r >= 0)) break;
    }
}

// Moves the ray-unordered segments of kModeTemp to their ray's CSR rows
// (fill[] zeroed, one counter per ray) ...
__global__ void __launch_bounds__(256) k_seg_scatter(const nif_segment* __restrict__ temp, const uint32_t* __restrict__ n_temp,
                                                     int64_t temp_cap, const uint32_t* __restrict__ offsets,
                                                     uint32_t* __restrict__ fill, nif_segment* __restrict__ segs,
                                                     int64_t cap, int n_rays) {
    int64_t n = *n_temp;
    if (n > temp_cap) n = temp_cap;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        nif_segment sg = temp[i];
        if (!NIF_IN(sg.ray, n_rays)) continue;
        int64_t g = (int64_t)offsets[sg.ray] + atomicAdd(fill + sg.ray, 1u);
        if (g < cap && NIF_IN(g, (int64_t)offsets[sg.ray + 1])) segs[g] = sg;
    }
}

// ... and sorts every ray's row by (t0, voxel). A warp takes 32 consecutive
// rays, whose rows are one contiguous range of at most kSortCap segments:
// lane l loads elements l, l + 32, ... of the range (coalesced) into
// registers and their keys into shared memory. Each element, not each row,
// then belongs to a lane, which counts the elements of the element's row
// that precede it (smaller (t0, voxel), ties by position: the stable order
// an insertion sort gives) and stores the element at that rank. A row of n
// costs n^2 compares spread over the warp's lanes, instead of n^2/2 serial
// steps on one lane while the others wait for the longest row. A longer
// range is sorted in place in global memory.
constexpr int kSortCap = 256;
constexpr int kSortPer = kSortCap / 32;

__global__ void __launch_bounds__(256) k_seg_sort(const uint32_t* __restrict__ offsets, int n_rays,
                                                  nif_segment* __restrict__ segs, int64_t cap) {
    __shared__ float2 s_key[8][kSortCap];           // (t0, voxel bits) of each element
    __shared__ uint8_t s_row[8][kSortCap];          // the warp-local row (lane) of each element
    __shared__ uint16_t s_beg[8][33];               // row bounds, relative to the range
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int r0 = (blockIdx.x * 8 + warp) * 32;
    if (r0 >= n_rays) return;
    const int r = r0 + lane;
    const int r1 = r0 + 32 < n_rays ? r0 + 32 : n_rays;
    auto clampc = [&](int64_t v) { return v < cap ? v : cap; };
    const int64_t b = clampc(offsets[r0]), e = clampc(offsets[r1]);
    const int64_t mb = r < n_rays ? clampc(offsets[r]) : e;
    const int64_t me = r < n_rays ? clampc(offsets[r + 1]) : e;
    const int len = (int)(e - b);
    if (len > kSortCap) {
        sort_row_inplace(segs, mb, me);
        return;
    }
    nif_segment el[kSortPer];
#pragma unroll
    for (int k = 0; k < kSortPer; k++) {
        const int i = lane + 32 * k;
        if (i < len) {
            el[k] = segs[b + i];
            s_key[warp][i] = make_float2(el[k].t0, __uint_as_float(el[k].voxel));
        }
    }
    s_beg[warp][lane] = (uint16_t)(mb - b);
    if (lane == 31) s_beg[warp][32] = (uint16_t)len;
    for (int i = (int)(mb - b); i < (int)(me - b); i++) s_row[warp][i] = (uint8_t)lane;
    __syncwarp();
#pragma unroll
    for (int k = 0; k < kSortPer; k++) {
        const int i = lane + 32 * k;
        if (i >= len) break;
        const int row = s_row[warp][i];
        const int j0 = s_beg[warp][row], j1 = s_beg[warp][row + 1];
        const float t = el[k].t0;
        const uint32_t v = el[k].voxel;
        int rank = 0;
        for (int j = j0; j < j1; j++) {
            const float2 o = s_key[warp][j];
            const uint32_t ov = __float_as_uint(o.y);
            rank += (o.x < t || (o.x == t && (ov < v || (ov == v && j < i)))) ? 1 : 0;
        }
        segs[b + j0 + rank] = el[k];
    }
}

// ---------------------------------------------------------------------------
// Exclusive scan of uint32 (three passes, 1024 elements per block)
// ---------------------------------------------------------------------------
constexpr int kScanT = 256, kScanE = 4, kScanB = kScanT * kScanE;
static_assert(kScanB == NIF_SCAN_BLOCK, "block-sum sizes of the scan's callers use NIF_SCAN_BLOCK");

__device__ __forceinline__ uint32_t block_excl_scan(uint32_t v, uint32_t* sh, uint32_t& total) {
    int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    uint32_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) sh[wid] = x;
    __syncthreads();
    if (wid == 0) {
        uint32_t w = lane < (int)(blockDim.x >> 5) ? sh[lane] : 0u;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t y = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += y;
        }
        sh[lane] = w;
    }
    __syncthreads();
    uint32_t warp_pre = wid > 0 ? sh[wid - 1] : 0u;
    total = sh[(blockDim.x >> 5) - 1];
    __syncthreads();
    return warp_pre + x - v;
}

__global__ void __launch_bounds__(kScanT) k_scan_blocks(const uint32_t* __restrict__ in, uint32_t* __restrict__ out,
                                                        uint32_t* __restrict__ bsum, int n) {
    __shared__ uint32_t sh[32];
    int64_t base = (int64_t)blockIdx.x * kScanB + threadIdx.x * kScanE;
    uint32_t v[kScanE], s = 0;
#pragma unroll
    for (int e = 0; e < kScanE; e++) {
        v[e] = base + e < n ? in[base + e] : 0u;
        s += v[e];
    }
    uint32_t total;
    uint32_t pre = block_excl_scan(s, sh, total);
#pragma unroll
    for (int e = 0; e < kScanE; e++) {
        if (base + e < n) out[base + e] = pre;
        pre += v[e];
    }
    if (threadIdx.x == 0) bsum[blockIdx.x] = total;
}

__global__ void __launch_bounds__(1024) k_scan_bsum(uint32_t* bsum, int nb, uint32_t* out_total) {
    __shared__ uint32_t sh[32];
    uint32_t carry = 0;
    for (int b0 = 0; b0 < nb; b0 += 1024) {
        int i = b0 + threadIdx.x;
        uint32_t v = i < nb ? bsum[i] : 0u;
        uint32_t total;
        uint32_t pre = block_excl_scan(v, sh, total);
        if (i < nb) bsum[i] = carry + pre;
        carry += total;
    }
    if (threadIdx.x == 0) *out_total = carry;
}

__global__ void __launch_bounds__(kScanT) k_scan_add(uint32_t* __restrict__ out, const uint32_t* __restrict__ bsum,
                                                     int n) {
    int64_t base = (int64_t)blockIdx.x * kScanB + threadIdx.x * kScanE;
    uint32_t add = bsum[blockIdx.x];
#pragma unroll
    for (int e = 0; e < kScanE; e++)
        if (base + e < n) out[base + e] += add;
}

__global__ void k_clamp_count(const uint32_t* offsets, int n_rays, int64_t cap, uint32_t* n_out,
                              int* status, int latch, int whole_rays) {
    uint32_t tot = offsets[n_rays];
    if ((int64_t)tot > cap) {
        if (latch) nif_set_status(status, NIF_ERR_CAPACITY);
        if (whole_rays) {          // the longest prefix of complete rows: largest offsets[r] <= cap
            int lo = 0, hi = n_rays;
            while (lo < hi) {
                int mid = (lo + hi + 1) >> 1;
                if ((int64_t)offsets[mid] <= cap) lo = mid; else hi = mid - 1;
            }
            tot = offsets[lo];
        } else {
            tot = (uint32_t)cap;
        }
    }
    *n_out = tot;
}

// ---------------------------------------------------------------------------
// Linearization
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_linearize(const nif_ray* __restrict__ rays, const int* __restrict__ inst_off,
                                                   int n_inst, const float4* __restrict__ poses, FieldView f,
                                                   const nif_segment* __restrict__ segs,
                                                   const uint32_t* __restrict__ n_dev, int64_t n_max,
                                                   nif_linseg* __restrict__ lin) {
    int64_t n = n_dev ? (int64_t)*n_dev : n_max;
    if (n > n_max) n = n_max;
    for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < n;
         s += (int64_t)gridDim.x * blockDim.x) {
        nif_segment sg = segs[s];
        const float4* R = reinterpret_cast<const float4*>(rays + sg.ray);
        float4 a = R[0], b = R[1];
        int inst = find_inst(inst_off, n_inst, (int)sg.ray);
        float4 pose = poses[inst];
        float3 x0 = make_float3(a.x + sg.t0 * a.w, a.y + sg.t0 * b.x, a.z + sg.t0 * b.y);
        float3 x1 = make_float3(a.x + sg.t1 * a.w, a.y + sg.t1 * b.x, a.z + sg.t1 * b.y);
        float3 p0 = nif_inverse(x0, pose);
        float3 p1 = nif_inverse(x1, pose);
        if (f.d && inst < f.n) {          // then p + u(p) = q by Newton
            p0 = nif_field_inverse(f, inst, p0);
            p1 = nif_field_inverse(f, inst, p1);
        }
        float dn = sqrtf(a.w * a.w + b.x * b.x + b.y * b.y);
        float dx = p1.x - p0.x, dy = p1.y - p0.y, dz = p1.z - p0.z;
        float4* L4 = reinterpret_cast<float4*>(lin + s);
        L4[0] = make_float4(p0.x, p0.y, p0.z, p1.x);
        L4[1] = make_float4(p1.y, p1.z, (sg.t1 - sg.t0) * dn, sqrtf(dx * dx + dy * dy + dz * dz));
    }
}

}  // namespace

// ---------------------------------------------------------------------------
// Launchers
// ---------------------------------------------------------------------------
nif_status nif_refit_run(nif_handle* h, int n_inst, cudaStream_t s) {
    NifProf prof_(h, "refit", s);
    if (h->n_leaves == 0) return NIF_OK;
    int64_t nl = (int64_t)h->n_leaves * n_inst;
    k_refit_leaves<<<nif_blocks(nl, 128), 128, 0, s>>>(h->N, h->n_leaves, h->n_nodes, n_inst, h->d_leaf_lat,
                                                      h->d_pose, nif_field_view(h), h->d_corners, h->d_aabb);
    NIF_CK_LAUNCH(h);
    for (size_t l = 0; l < h->level_begin.size(); l++) {
        int64_t nn = (int64_t)h->level_count[l] * n_inst;
        k_refit_level<<<nif_blocks(nn, 128), 128, 0, s>>>(h->level_begin[l], h->level_count[l], h->n_leaves,
                                                         h->n_nodes, n_inst, h->d_child, h->d_aabb);
        NIF_CK_LAUNCH(h);
    }
    return NIF_OK;
}

static TreeView tree_view(nif_handle* h);

// warps per traversal block: a tuning knob of the handle (2, 4 or 8); the
// count and temp modes run the persistent kernel (grid: 32 warps per SM)
template <int MODE, int W, bool BIL = false>
static void launch_traverse_w(nif_handle* h, const nif_ray* rays, const int* inst_off, int n_inst, int n_rays,
                              uint32_t* counts, const uint32_t* offsets, nif_segment* segs, int64_t cap,
                              uint32_t* cursor, cudaStream_t s, int64_t emit_skip_le) {
    const TreeView tv = tree_view(h);
    if (MODE == kModeEmit) {
        k_seg_traverse<kModeEmit, W, BIL><<<nif_blocks(n_rays, 32 * W), 32 * W, 0, s>>>(
            rays, inst_off, n_inst, n_rays, tv, h->d_corners, h->d_aabb, counts, offsets, segs, cap, cursor,
            emit_skip_le, h->d_status);
        return;
    }
    cudaMemsetAsync(h->d_next, 0, sizeof(uint32_t), s);
    const unsigned grid = std::min<unsigned>(nif_blocks(n_rays, 32 * W), (unsigned)h->num_sms * (32 / W));
    constexpr int M = MODE == kModeTemp ? kModeTemp : kModeCount;
    k_seg_traverse_p<M, W, BIL><<<grid, 32 * W, 0, s>>>(rays, inst_off, n_inst, n_rays, tv, h->d_corners,
                                                        h->d_aabb, counts, segs, cap, cursor, h->d_next,
                                                        h->d_status);
}

template <int MODE>
static void launch_traverse(nif_handle* h, const nif_ray* rays, const int* inst_off, int n_inst, int n_rays,
                            uint32_t* counts, const uint32_t* offsets, nif_segment* segs, int64_t cap,
                            uint32_t* cursor, cudaStream_t s, int64_t emit_skip_le = 0) {
    if (h->cfg.flags & NIF_FLAG_BILINEAR_FACES) {   // one block size for the curved-face variant
        launch_traverse_w<MODE, 4, true>(h, rays, inst_off, n_inst, n_rays, counts, offsets, segs, cap, cursor, s,
                                         emit_skip_le);
        return;
    }
    switch (h->tune.trav_warps) {
        case 2:
            launch_traverse_w<MODE, 2>(h, rays, inst_off, n_inst, n_rays, counts, offsets, segs, cap, cursor, s,
                                       emit_skip_le);
            break;
        case 8:
            launch_traverse_w<MODE, 8>(h, rays, inst_off, n_inst, n_rays, counts, offsets, segs, cap, cursor, s,
                                       emit_skip_le);
            break;
        default:
            launch_traverse_w<MODE, 4>(h, rays, inst_off, n_inst, n_rays, counts, offsets, segs, cap, cursor, s,
                                       emit_skip_le);
    }
}

static TreeView tree_view(nif_handle* h) {
    TreeView t;
    t.n_leaves = h->n_leaves;
    t.n_nodes = h->n_nodes;
    t.top_begin = h->top_begin;
    t.top_count = h->top_count;
    t.child = h->d_child;
    t.leaf_vox = h->d_leaf_vox;
    return t;
}

// Exit-face walk (k_seg_walk): the deformed lattice of every instance (the
// handle's current poses), the voxel -> leaf map on first use, then one walk
// launch. mode: 0 counts, 1 emits into `offsets` rows, 2 first BVH query only.
nif_status nif_seg_walk_run(nif_handle* h, const nif_ray* rays, const int* inst_off, int n_inst, int n_rays,
                            uint32_t* counts, const uint32_t* offsets, nif_segment* segs, int64_t cap, int mode,
                            cudaStream_t s) {
    if (n_rays <= 0) return NIF_OK;
    if (h->n_leaves == 0) {
        if (mode != 1) NIF_CK(h, cudaMemsetAsync(counts, 0, sizeof(uint32_t) * n_rays, s));
        return NIF_OK;
    }
    nif_status st;
    if (mode != 2) {
        NifProf prof_(h, "walk_lattice", s);
        const int64_t M = h->N + 1, per = M * M * M;
        if ((st = nif_grow(h, h->b_lattice, sizeof(float4) * (size_t)(per * n_inst))) != NIF_OK) return st;
        k_lattice<<<nif_blocks(per * n_inst, 256), 256, 0, s>>>(h->N, n_inst, h->d_pose, nif_field_view(h),
                                                               (float4*)h->b_lattice.p);
        NIF_CK_LAUNCH(h);
        if (!h->d_vox_leaf) {
            const size_t nv = (size_t)h->N * h->N * h->N;
            NIF_CK(h, cudaMalloc(&h->d_vox_leaf, sizeof(int) * nv));
            NIF_CK(h, cudaMemsetAsync(h->d_vox_leaf, 0xFF, sizeof(int) * nv, s));
            k_vox_leaf<<<nif_blocks(h->n_leaves, 256), 256, 0, s>>>(h->d_leaf_vox, h->n_leaves, h->d_vox_leaf);
            NIF_CK_LAUNCH(h);
        }
    }
    const TreeView tv = tree_view(h);
    const float4* lat = (const float4*)h->b_lattice.p;
    const unsigned g = nif_blocks(n_rays, 128);
    if (mode == 0) {
        NifProf prof_(h, "walk_count", s);
        k_seg_walk<kWalkCount><<<g, 128, 0, s>>>(rays, inst_off, n_inst, n_rays, h->N, tv, h->d_corners, h->d_aabb,
                                                 lat, h->d_vox_leaf, counts, nullptr, nullptr, 0, h->d_status);
    } else if (mode == 1) {
        NifProf prof_(h, "walk_emit", s);
        k_seg_walk<kWalkEmit><<<g, 128, 0, s>>>(rays, inst_off, n_inst, n_rays, h->N, tv, h->d_corners, h->d_aabb,
                                                lat, h->d_vox_leaf, nullptr, offsets, segs, cap, h->d_status);
    } else {
        NifProf prof_(h, "walk_first", s);
        k_seg_walk<kWalkFirst><<<g, 128, 0, s>>>(rays, inst_off, n_inst, n_rays, h->N, tv, h->d_corners, h->d_aabb,
                                                 lat, h->d_vox_leaf, counts, nullptr, nullptr, 0, h->d_status);
    }
    NIF_CK_LAUNCH(h);
    return NIF_OK;
}

nif_status nif_seg_count_run(nif_handle* h, const nif_ray* rays, const int* inst_off, int n_inst, int n_rays,
                             uint32_t* counts, cudaStream_t s) {
    NifProf prof_(h, "seg_count", s);
    if (n_rays <= 0) return NIF_OK;
    if (h->n_leaves == 0) {
        NIF_CK(h, cudaMemsetAsync(counts, 0, sizeof(uint32_t) * n_rays, s));
        return NIF_OK;
    }
    launch_traverse<kModeCount>(h, rays, inst_off, n_inst, n_rays, counts, nullptr, nullptr, 0, nullptr, s);
    NIF_CK_LAUNCH(h);
    return NIF_OK;
}

nif_status nif_seg_emit_run(nif_handle* h, const nif_ray* rays, const int* inst_off, int n_inst, int n_rays,
                            const uint32_t* offsets, nif_segment* segs, int64_t cap, cudaStream_t s) {
    NifProf prof_(h, "seg_emit", s);
    if (n_rays <= 0 || h->n_leaves == 0) return NIF_OK;
    launch_traverse<kModeEmit>(h, rays, inst_off, n_inst, n_rays, nullptr, offsets, segs, cap, nullptr, s);
    NIF_CK_LAUNCH(h);
    return NIF_OK;
}

nif_status nif_seg_emit_if_overflow_run(nif_handle* h, const nif_ray* rays, const int* inst_off, int n_inst, int n_rays,
                                        const uint32_t* offsets, nif_segment* segs, int64_t cap,
                                        uint32_t* temp_cursor, int64_t temp_cap, cudaStream_t s) {
    NifProf prof_(h, "seg_emit", s);
    if (n_rays <= 0 || h->n_leaves == 0) return NIF_OK;
    launch_traverse<kModeEmit>(h, rays, inst_off, n_inst, n_rays, nullptr, offsets, segs, cap, temp_cursor, s,
                               temp_cap);
    NIF_CK_LAUNCH(h);
    return NIF_OK;
}

// One traversal: per-ray counts and all segments, ray-unordered, into temp
// (capacity temp_cap; *cursor must be zero and ends as the total).
nif_status nif_seg_temp_run(nif_handle* h, const nif_ray* rays, const int* inst_off, int n_inst, int n_rays,
                            uint32_t* counts, nif_segment* temp, int64_t temp_cap, uint32_t* cursor,
                            cudaStream_t s) {
    NifProf prof_(h, "seg_traverse", s);
    if (n_rays <= 0) return NIF_OK;
    if (h->n_leaves == 0) {
        NIF_CK(h, cudaMemsetAsync(counts, 0, sizeof(uint32_t) * n_rays, s));
        return NIF_OK;
    }
    launch_traverse<kModeTemp>(h, rays, inst_off, n_inst, n_rays, counts, nullptr, temp, temp_cap, cursor, s);
    NIF_CK_LAUNCH(h);
    return NIF_OK;
}

// temp -> CSR rows in ray order, then each row sorted; fill must hold n_rays zeroed words
nif_status nif_seg_scatter_run(nif_handle* h, const nif_segment* temp, const uint32_t* n_temp,
                               int64_t n_temp_max, const uint32_t* offsets, uint32_t* fill, int n_rays,
                               nif_segment* segs, int64_t cap, cudaStream_t s) {
    NifProf prof_(h, "seg_scatter", s);
    if (n_rays <= 0) return NIF_OK;
    unsigned g = nif_blocks(std::max<int64_t>(n_temp_max, 1), 256);
    unsigned gcap = (unsigned)h->num_sms * 8;
    if (g > gcap) g = gcap;
    k_seg_scatter<<<g, 256, 0, s>>>(temp, n_temp, n_temp_max, offsets, fill, segs, cap, n_rays);
    NIF_CK_LAUNCH(h);
    k_seg_sort<<<nif_blocks(n_rays, 256), 256, 0, s>>>(offsets, n_rays, segs, cap);   // 8 warps x 32 rays
    NIF_CK_LAUNCH(h);
    return NIF_OK;
}

nif_status nif_scan_run(nif_handle* h, const uint32_t* in, uint32_t* out, int n, cudaStream_t s) {
    NifProf prof_(h, "scan", s);
    int nb = (int)nif_blocks(n, kScanB);
    nif_status st = nif_grow(h, h->b_scan, sizeof(uint32_t) * (size_t)(nb + 1));
    if (st != NIF_OK) return st;
    uint32_t* bsum = (uint32_t*)h->b_scan.p;
    if (n > 0) {
        k_scan_blocks<<<nb, kScanT, 0, s>>>(in, out, bsum, n);
        NIF_CK_LAUNCH(h);
    }
    k_scan_bsum<<<1, 1024, 0, s>>>(bsum, n > 0 ? nb : 0, out + n);
    NIF_CK_LAUNCH(h);
    if (n > 0) {
        k_scan_add<<<nb, kScanT, 0, s>>>(out, bsum, n);
        NIF_CK_LAUNCH(h);
    }
    return NIF_OK;
}

nif_status nif_clamp_count_run(nif_handle* h, const uint32_t* offsets, int n_rays, int64_t cap, uint32_t* n_out,
                               bool latch, cudaStream_t s, bool whole_rays) {
    k_clamp_count<<<1, 1, 0, s>>>(offsets, n_rays, cap, n_out, h->d_status, latch ? 1 : 0, whole_rays ? 1 : 0);
    NIF_CK_LAUNCH(h);
    return NIF_OK;
}

nif_status nif_linearize_with_run(nif_handle* h, const nif_ray* rays, const int* inst_off, int n_inst,
                                  const float4* poses_dev, FieldView f, const nif_segment* segs,
                                  const uint32_t* n_dev, int64_t n_max, nif_linseg* lin, cudaStream_t s) {
    NifProf prof_(h, "linearize", s);
    if (n_max <= 0) return NIF_OK;
    unsigned g = nif_blocks(n_max, 256);
    unsigned cap = (unsigned)h->num_sms * 8;
    if (g > cap) g = cap;
    k_linearize<<<g, 256, 0, s>>>(rays, inst_off, n_inst, poses_dev, f, segs, n_dev, n_max, lin);
    NIF_CK_LAUNCH(h);
    return NIF_OK;
}

nif_status nif_linearize_run(nif_handle* h, const nif_ray* rays, const int* inst_off, int n_inst,
                             const nif_segment* segs, const uint32_t* n_dev, int64_t n_max, nif_linseg* lin,
                             cudaStream_t s) {
    return nif_linearize_with_run(h, rays, inst_off, n_inst, h->d_pose, nif_field_view(h), segs, n_dev, n_max, lin, s);
}

// Exclusive scan with caller-provided block-sum storage (at least
// ceil(n / 1024) + 1 words); allocates nothing.
nif_status nif_scan_run_with(nif_handle* h, const uint32_t* in, uint32_t* out, int n, uint32_t* bsum,
                             cudaStream_t s) {
    int nb = (int)nif_blocks(n, kScanB);
    if (n > 0) {
        k_scan_blocks<<<nb, kScanT, 0, s>>>(in, out, bsum, n);
        NIF_CK_LAUNCH(h);
    }
    k_scan_bsum<<<1, 1024, 0, s>>>(bsum, n > 0 ? nb : 0, out + n);
    NIF_CK_LAUNCH(h);
    if (n > 0) {
        k_scan_add<<<nb, kScanT, 0, s>>>(out, bsum, n);
        NIF_CK_LAUNCH(h);
    }
    return NIF_OK;
}
