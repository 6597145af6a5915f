// k_pose.cu -- gradient of a loss with respect to the deformation parameters
// (pose fitting). A segment's rest end points are p = D^-1(x; theta) of fixed
// deformed points x, so D(p(theta); theta) = x and, by the implicit function
// theorem, dp/dtheta = -J_D(p)^-1 dD/dtheta(p). Given dL/dp of both end
// points, each segment contributes -(J_D^-T dL/dp) . dD/dtheta_j to
// dL/dtheta_j of its instance.
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
                                                   const float4* __restrict__ poses, float* __restrict__ dposes) {
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

}  // namespace

nif_status nif_pose_grad_run(nif_handle* h, const nif_segment* segs, const nif_linseg* lin, const float* dp,
                             const uint32_t* n_dev, int64_t n, const int* inst_off, int n_inst, float* dposes,
                             cudaStream_t s) {
    NifProf prof_(h, "pose_grad", s);
    if (n <= 0) return NIF_OK;
    unsigned g = nif_blocks(n, 256);
    unsigned cap = (unsigned)h->num_sms * 8;
    if (g > cap) g = cap;
    k_pose_grad<<<g, 256, 0, s>>>(segs, lin, dp, n_dev, n, inst_off, n_inst, h->d_pose, dposes);
    NIF_CK_LAUNCH(h);
    return NIF_OK;
}
