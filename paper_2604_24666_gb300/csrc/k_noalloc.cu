// k_noalloc.cu -- segment generation that allocates no device memory.
//
// For callers that cannot call cudaMalloc: a host application that owns all
// device memory (an engine or renderer with its own fixed-budget allocator),
// or a latency-critical loop where cudaMalloc's implicit device-wide
// synchronisation is not acceptable. nif_segments itself grows per-handle
// scratch on demand; this variant keeps its scratch -- the per-ray counts and
// the scan's block sums -- in one file-scope device array of fixed size that
// every GPU loading the library holds until the process exits.
#include <mutex>

#include "nif_internal.cuh"

namespace {

constexpr int kMaxRays = NIF_NOALLOC_MAX_RAYS;
// the scan of kMaxRays counts needs one block sum per NIF_SCAN_BLOCK rays and the total
constexpr int kBlockSums = 2048;
static_assert(kBlockSums >= (kMaxRays + NIF_SCAN_BLOCK - 1) / NIF_SCAN_BLOCK + 1,
              "block-sum part of the static scratch too small for NIF_NOALLOC_MAX_RAYS");

// [0, kMaxRays): per-ray segment counts; [kMaxRays, +kBlockSums): scan block sums
static __device__ __align__(256) uint32_t g_noalloc_scratch[kMaxRays + kBlockSums];

constexpr int kMaxDevices = 64;
uint32_t* g_scratch_addr[kMaxDevices] = {nullptr};
std::mutex g_scratch_mtx;

// Device address of the static scratch on the current device (looked up once
// per device with that device current). The host-side symbol is only a
// stand-in and must never be handed to a kernel.
nif_status scratch_address(nif_handle* h, uint32_t** out) {
    int dev = -1;
    NIF_CK(h, cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) return nif_fail(h, NIF_ERR_ARG, "device index out of range");
    std::lock_guard<std::mutex> lock(g_scratch_mtx);
    if (!g_scratch_addr[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) return nif_cuda_fail(h, e, "cudaGetSymbolAddress(noalloc scratch)");
        g_scratch_addr[dev] = static_cast<uint32_t*>(p);
    }
    *out = g_scratch_addr[dev];
    return NIF_OK;
}

}  // namespace

extern "C" nif_status nif_segments_noalloc(nif_handle* h, const nif_pose* poses, int n_inst, const nif_ray* rays,
                                           const int* inst_off, int n_rays, uint32_t* ray_offsets,
                                           nif_segment* segs, int64_t seg_cap, int64_t* n_segs_host,
                                           void* stream) {
    if (!h) return NIF_ERR_ARG;
    nif_status st = nif_check_inst(h, poses, n_inst, inst_off, n_rays);
    if (st != NIF_OK) return st;
    if (n_rays > kMaxRays)
        return nif_fail(h, NIF_ERR_ARG, "nif_segments_noalloc: n_rays must be in [0, NIF_NOALLOC_MAX_RAYS]");
    // checked before nif_upload_poses, which would otherwise grow the
    // per-instance buffers: within inst_cap it allocates nothing
    if (n_inst > h->inst_cap)
        return nif_fail(h, NIF_ERR_ARG,
                        "nif_segments_noalloc: more instances than the handle holds buffers for "
                        "(an earlier allocating call with that many instances provides them)");
    if (!ray_offsets || (n_rays > 0 && !rays)) return nif_fail(h, NIF_ERR_ARG, "buffers");
    cudaStream_t s = (cudaStream_t)stream;
    uint32_t* scratch = nullptr;
    if ((st = scratch_address(h, &scratch)) != NIF_OK) return st;
    if ((st = nif_upload_poses(h, poses, n_inst, s)) != NIF_OK) return st;
    uint32_t* counts = scratch;
    uint32_t* bsum = scratch + kMaxRays;
    if ((st = nif_refit_run(h, n_inst, s)) != NIF_OK) return st;
    if ((st = nif_seg_count_run(h, rays, inst_off, n_inst, n_rays, counts, s)) != NIF_OK) return st;
    if ((st = nif_scan_run_with(h, counts, ray_offsets, n_rays, bsum, s)) != NIF_OK) return st;
    if (segs && (st = nif_seg_emit_run(h, rays, inst_off, n_inst, n_rays, ray_offsets, segs, seg_cap, s)) != NIF_OK)
        return st;
    NIF_CK(h, cudaStreamSynchronize(s));
    uint32_t tot = 0;
    NIF_CK(h, cudaMemcpy(&tot, ray_offsets + n_rays, sizeof(uint32_t), cudaMemcpyDeviceToHost));
    if (n_segs_host) *n_segs_host = tot;
    if ((st = nif_check_status(h, s)) != NIF_OK) return st;
    if (segs && (int64_t)tot > seg_cap) return nif_fail(h, NIF_ERR_CAPACITY, "segment capacity exceeded");
    return NIF_OK;
}
