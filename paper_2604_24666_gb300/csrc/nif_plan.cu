// nif_plan.cu -- batched query of many deforming instances as one CUDA graph.
//
// A plan fixes the caller's buffers (rays, instance offsets, hits), the
// segment capacity and the launch knobs, runs the whole query path once per
// knob setting to pick the fastest (coordinate descent over traversal warps
// per block, encoding block size and grid, and rows per encode + MLP chunk),
// and captures the path into a CUDA graph. Every stage after the pose upload
// reads its element counts from device memory (segment totals, per-chunk
// counts), so one replay needs no host round trip: the host only writes the
// new poses into a pinned buffer and launches the graph.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "nif_internal.cuh"

struct nif_query_plan {
    nif_handle* h = nullptr;
    int n_inst = 0, n_rays = 0;
    const nif_ray* rays = nullptr;
    const int* inst_off = nullptr;
    nif_hit* hits = nullptr;
    unsigned flags = 0;
    int64_t cap = 0;             // segment capacity
    int64_t chunk = 0;           // rows per encode + MLP chunk
    int n_chunks = 0;
    float4* pinned_poses = nullptr;
    uint32_t* chunk_counts = nullptr;
    cudaStream_t cap_stream = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaEvent_t done = nullptr;
    bool launched = false;
    bool counted = false;        // holds a place in the handle's live-plan count
};

namespace {

__global__ void k_chunk_counts(const uint32_t* __restrict__ n_dev, int64_t chunk, int n_chunks,
                               uint32_t* __restrict__ counts) {
    int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= n_chunks) return;
    int64_t rem = (int64_t)*n_dev - (int64_t)c * chunk;
    counts[c] = (uint32_t)(rem <= 0 ? 0 : (rem < chunk ? rem : chunk));
}

}  // namespace

nif_status nif_chunk_counts_run(nif_handle* h, const uint32_t* n_dev, int64_t chunk, int n_chunks, uint32_t* counts,
                                cudaStream_t s) {
    if (n_chunks <= 0) return NIF_OK;
    k_chunk_counts<<<nif_blocks(n_chunks, 128), 128, 0, s>>>(n_dev, chunk, n_chunks, counts);
    NIF_CK_LAUNCH(h);
    return NIF_OK;
}

namespace {

void write_poses(nif_query_plan* p, const nif_pose* poses) {
    for (int i = 0; i < p->n_inst; i++)
        p->pinned_poses[i] = make_float4(NIF_KBEND * poses[i].bend, poses[i].twist, poses[i].taper, 0.f);
}

// The whole query path with device-side counts (no host synchronisation).
nif_status plan_enqueue(nif_query_plan* p, cudaStream_t s) {
    nif_handle* h = p->h;
    nif_status st;
    const int n = p->n_rays;
    uint32_t* counts = (uint32_t*)h->b_counts.p;
    uint32_t* offs = (uint32_t*)h->b_offsets.p;
    uint32_t* n_dev = offs + n + 1;
    uint32_t* cursor = reinterpret_cast<uint32_t*>(h->d_count + 1);
    nif_segment* temp = (nif_segment*)h->b_temp.p;
    nif_segment* segs = (nif_segment*)h->b_segs.p;
    nif_linseg* lin = (nif_linseg*)h->b_lin.p;
    float* out = (float*)h->b_out.p;
    NIF_CK(h, cudaMemcpyAsync(h->d_pose, p->pinned_poses, sizeof(float4) * p->n_inst, cudaMemcpyHostToDevice, s));
    if ((st = nif_refit_run(h, p->n_inst, s)) != NIF_OK) return st;
    NIF_CK(h, cudaMemsetAsync(cursor, 0, sizeof(uint32_t), s));
    if ((st = nif_seg_temp_run(h, p->rays, p->inst_off, p->n_inst, n, counts, temp, p->cap, cursor, s)) != NIF_OK)
        return st;
    if ((st = nif_scan_run(h, counts, offs, n, s)) != NIF_OK) return st;
    if ((st = nif_clamp_count_run(h, offs, n, p->cap, n_dev, true, s)) != NIF_OK) return st;
    NIF_CK(h, cudaMemsetAsync(counts, 0, sizeof(uint32_t) * (size_t)n, s));
    if ((st = nif_seg_scatter_run(h, temp, cursor, p->cap, offs, counts, n, segs, p->cap, s)) != NIF_OK) return st;
    if ((st = nif_linearize_run(h, p->rays, p->inst_off, p->n_inst, segs, n_dev, p->cap, lin, s)) != NIF_OK) return st;
    const int prec = h->cfg.precision;
    if (prec != NIF_FP32 && nif_mlp_enc_fusable(h)) {
        // encoding and MLP in one launch over every segment: no feature matrix
        if ((st = nif_mlp_enc_tc_run(h, lin, n_dev, p->cap, out, s)) != NIF_OK) return st;
        return nif_reconstruct_run(h, p->rays, p->inst_off, p->n_inst, n, offs, segs, p->cap, lin, out, p->hits,
                                   p->flags, s);
    }
    if ((st = nif_chunk_counts_run(h, n_dev, p->chunk, p->n_chunks, p->chunk_counts, s)) != NIF_OK) return st;
    for (int c = 0; c < p->n_chunks; c++) {
        int64_t c0 = (int64_t)c * p->chunk;
        int64_t len = std::min(p->chunk, p->cap - c0);
        const uint32_t* cn = p->chunk_counts + c;
        if (prec == NIF_FP32) {
            if ((st = nif_encode_segments_run(h, lin + c0, cn, len, h->b_feat.p, NIF_FP32, NIF_FP32, s)) != NIF_OK)
                return st;
            if ((st = nif_mlp_fwd_fp32_run(h, (const float*)h->b_feat.p, cn, len, out + c0 * NIF_OUT,
                                           (float*)h->b_acts.p, s, 0, true)) != NIF_OK)
                return st;
        } else {
            if ((st = nif_encode_segments_run(h, lin + c0, cn, len, h->b_feat.p, prec, NIF_FP16, s)) != NIF_OK)
                return st;
            if ((st = nif_mlp_fwd_tc_run(h, h->b_feat.p, prec, cn, len, out + c0 * NIF_OUT, s)) != NIF_OK) return st;
        }
    }
    return nif_reconstruct_run(h, p->rays, p->inst_off, p->n_inst, n, offs, segs, p->cap, lin, out, p->hits, p->flags,
                               s);
}

// (Re)size the chunking and the buffers it needs.
nif_status plan_buffers(nif_query_plan* p, int64_t chunk) {
    nif_handle* h = p->h;
    nif_status st;
    p->chunk = std::max<int64_t>(1, std::min(chunk, p->cap));
    p->n_chunks = (int)((p->cap + p->chunk - 1) / p->chunk);
    size_t esz = h->cfg.precision == NIF_FP32 ? 4 : 2;
    if ((st = nif_grow(h, h->b_feat, esz * (size_t)h->in_dim * p->chunk)) != NIF_OK) return st;
    if (h->cfg.precision == NIF_FP32 &&
        (st = nif_grow(h, h->b_acts, sizeof(float) * (size_t)p->chunk * h->W * h->H)) != NIF_OK)
        return st;
    if (p->chunk_counts) cudaFree(p->chunk_counts);
    p->chunk_counts = nullptr;
    NIF_CK(h, cudaMalloc(&p->chunk_counts, sizeof(uint32_t) * p->n_chunks));
    return NIF_OK;
}

nif_status time_once(nif_query_plan* p, cudaStream_t s, float* ms) {
    nif_handle* h = p->h;
    cudaEvent_t a, b;
    NIF_CK(h, cudaEventCreate(&a));
    NIF_CK(h, cudaEventCreate(&b));
    nif_status st = plan_enqueue(p, s);   // warm
    if (st == NIF_OK) {
        cudaEventRecord(a, s);
        st = plan_enqueue(p, s);
        cudaEventRecord(b, s);
    }
    if (st == NIF_OK) {
        cudaEventSynchronize(b);
        cudaEventElapsedTime(ms, a, b);
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    return st;
}

nif_status autotune(nif_query_plan* p, cudaStream_t s) {
    nif_handle* h = p->h;
    nif_status st;
    float best = 0.f;
    if ((st = time_once(p, s, &best)) != NIF_OK) return st;
    auto try_knob = [&](int* knob, const std::vector<int>& values) -> nif_status {
        int keep = *knob;
        for (int v : values) {
            if (v == keep) continue;
            *knob = v;
            float ms = 0.f;
            nif_status e = time_once(p, s, &ms);
            if (e != NIF_OK) return e;
            if (ms < best) { best = ms; keep = v; }
        }
        *knob = keep;
        return NIF_OK;
    };
    if (nif_mlp_enc_fusable(h) && (st = try_knob(&h->tune.query_fused, {0, 1})) != NIF_OK) return st;
    if (h->cfg.precision == NIF_FP32 && (st = try_knob(&h->tune.query_fp32_fused, {0, 1})) != NIF_OK) return st;
    if ((st = try_knob(&h->tune.trav_warps, {2, 4, 8})) != NIF_OK) return st;
    if ((st = try_knob(&h->tune.enc_threads, {128, 256, 512})) != NIF_OK) return st;
    if ((st = try_knob(&h->tune.enc_blocks_per_sm, {4, 8, 16, 32})) != NIF_OK) return st;
    if (h->cfg.precision != NIF_FP32) {
        int64_t keep = h->tune.tc_chunk;
        for (int64_t c : {(int64_t)1 << 18, (int64_t)1 << 19, (int64_t)1 << 20, (int64_t)1 << 21}) {
            if (c == keep) continue;
            if ((st = plan_buffers(p, c)) != NIF_OK) return st;
            float ms = 0.f;
            if ((st = time_once(p, s, &ms)) != NIF_OK) return st;
            if (ms < best) { best = ms; keep = c; }
        }
        h->tune.tc_chunk = keep;
        if ((st = plan_buffers(p, keep)) != NIF_OK) return st;
    }
    return NIF_OK;
}

}  // namespace

extern "C" nif_status nif_query_plan_create(nif_handle* h, int n_inst, const nif_ray* rays, const int* inst_off,
                                            int n_rays, nif_hit* hits, int64_t seg_capacity, unsigned flags,
                                            int autotune_flag, const nif_pose* poses, nif_query_plan** out) {
    if (!h || !out) return NIF_ERR_ARG;
    *out = nullptr;
    if (!poses || n_inst < 1 || n_rays < 1 || !rays || !hits || (n_inst > 1 && !inst_off))
        return nif_fail(h, NIF_ERR_ARG, "query plan arguments");
    nif_status st;
    nif_query_plan* p = new nif_query_plan();
    auto fail = [&](nif_status e) {
        nif_query_plan_destroy(p);
        return e;
    };
    p->h = h;
    p->n_inst = n_inst;
    p->n_rays = n_rays;
    p->rays = rays;
    p->inst_off = inst_off;
    p->hits = hits;
    p->flags = flags;
    if (cudaStreamCreateWithFlags(&p->cap_stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&p->done, cudaEventDisableTiming) != cudaSuccess ||
        cudaMallocHost(&p->pinned_poses, sizeof(float4) * n_inst) != cudaSuccess)
        return fail(nif_fail(h, NIF_ERR_CUDA, "plan stream / event / pinned buffer"));
    cudaStream_t s = p->cap_stream;
    if ((st = nif_ensure_instances(h, n_inst)) != NIF_OK) return fail(st);
    write_poses(p, poses);
    if ((st = nif_grow(h, h->b_counts, sizeof(uint32_t) * ((size_t)n_rays + 1))) != NIF_OK) return fail(st);
    if ((st = nif_grow(h, h->b_offsets, sizeof(uint32_t) * ((size_t)n_rays + 2))) != NIF_OK) return fail(st);
    // capacity: measured segments of the given poses with a margin, unless given
    if (seg_capacity <= 0) {
        NIF_CK(h, cudaMemcpyAsync(h->d_pose, p->pinned_poses, sizeof(float4) * n_inst, cudaMemcpyHostToDevice, s));
        if ((st = nif_refit_run(h, n_inst, s)) != NIF_OK) return fail(st);
        uint32_t* counts = (uint32_t*)h->b_counts.p;
        uint32_t* offs = (uint32_t*)h->b_offsets.p;
        if ((st = nif_seg_count_run(h, rays, inst_off, n_inst, n_rays, counts, s)) != NIF_OK) return fail(st);
        if ((st = nif_scan_run(h, counts, offs, n_rays, s)) != NIF_OK) return fail(st);
        uint32_t tot = 0;
        NIF_CK(h, cudaStreamSynchronize(s));
        NIF_CK(h, cudaMemcpy(&tot, offs + n_rays, sizeof(uint32_t), cudaMemcpyDeviceToHost));
        seg_capacity = std::max<int64_t>(1024, (int64_t)(tot * 1.5) + 1024);
    }
    p->cap = seg_capacity;
    if ((st = nif_grow(h, h->b_temp, sizeof(nif_segment) * (size_t)p->cap)) != NIF_OK) return fail(st);
    if ((st = nif_grow(h, h->b_segs, sizeof(nif_segment) * (size_t)p->cap)) != NIF_OK) return fail(st);
    if ((st = nif_grow(h, h->b_lin, sizeof(nif_linseg) * (size_t)p->cap)) != NIF_OK) return fail(st);
    if ((st = nif_grow(h, h->b_out, sizeof(float) * NIF_OUT * (size_t)p->cap)) != NIF_OK) return fail(st);
    if ((st = nif_grow(h, h->b_scan, sizeof(uint32_t) * (size_t)(nif_blocks(n_rays, 1024) + 1))) != NIF_OK)
        return fail(st);
    int64_t chunk = h->tune.tc_chunk;
    if ((st = plan_buffers(p, chunk)) != NIF_OK) return fail(st);
    if ((st = h->cfg.precision == NIF_FP32 ? nif_refresh_x3(h, s) : nif_refresh_lowp(h, s)) != NIF_OK) return fail(st);
    bool prof = h->prof;
    h->prof = false;
    if (autotune_flag && (st = autotune(p, s)) != NIF_OK) { h->prof = prof; return fail(st); }
    // one uncaptured run settles every lazily set attribute before capture
    if ((st = plan_enqueue(p, s)) != NIF_OK) { h->prof = prof; return fail(st); }
    NIF_CK(h, cudaStreamSynchronize(s));
    NIF_CK(h, cudaStreamBeginCapture(s, cudaStreamCaptureModeRelaxed));
    st = plan_enqueue(p, s);
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamEndCapture(s, &g);
    h->prof = prof;
    if (st != NIF_OK) { if (g) cudaGraphDestroy(g); return fail(st); }
    if (e != cudaSuccess) return fail(nif_cuda_fail(h, e, "cudaStreamEndCapture"));
    p->graph = g;
    e = cudaGraphInstantiate(&p->exec, g, 0);
    if (e != cudaSuccess) return fail(nif_cuda_fail(h, e, "cudaGraphInstantiate"));
    p->counted = true;
    h->n_plans++;
    *out = p;
    return NIF_OK;
}

extern "C" nif_status nif_query_plan_run(nif_query_plan* p, const nif_pose* poses, void* stream) {
    if (!p || !poses) return NIF_ERR_ARG;
    nif_handle* h = p->h;
    for (int i = 0; i < p->n_inst; i++)
        if (!(std::fabs(poses[i].bend) <= 1.0f && std::fabs(poses[i].twist) <= 4.0f && std::fabs(poses[i].taper) <= 1.0f))
            return nif_fail(h, NIF_ERR_ARG, "pose outside |bend| <= 1, |twist| <= 4, |taper| <= 1");
    cudaStream_t s = (cudaStream_t)stream;
    // the previous replay must have consumed the pinned poses before they change
    if (p->launched) NIF_CK(h, cudaEventSynchronize(p->done));
    write_poses(p, poses);
    nif_status st = h->cfg.precision == NIF_FP32 ? nif_refresh_x3(h, s) : nif_refresh_lowp(h, s);
    if (st != NIF_OK) return st;
    NIF_CK(h, cudaGraphLaunch(p->exec, s));
    NIF_CK(h, cudaEventRecord(p->done, s));
    p->launched = true;
    return NIF_OK;
}

extern "C" nif_status nif_query_plan_info(const nif_query_plan* p, int* trav_warps, int* enc_threads,
                                          int* enc_blocks_per_sm, int64_t* tc_chunk, int64_t* seg_capacity) {
    if (!p) return NIF_ERR_ARG;
    if (trav_warps) *trav_warps = p->h->tune.trav_warps;
    if (enc_threads) *enc_threads = p->h->tune.enc_threads;
    if (enc_blocks_per_sm) *enc_blocks_per_sm = p->h->tune.enc_blocks_per_sm;
    if (tc_chunk) *tc_chunk = p->chunk;
    if (seg_capacity) *seg_capacity = p->cap;
    return NIF_OK;
}

extern "C" void nif_query_plan_destroy(nif_query_plan* p) {
    if (!p) return;
    if (p->cap_stream) cudaStreamSynchronize(p->cap_stream);
    if (p->done && p->launched) cudaEventSynchronize(p->done);
    if (p->counted && --p->h->n_plans == 0) nif_free_retired(p->h);
    if (p->exec) cudaGraphExecDestroy(p->exec);
    if (p->graph) cudaGraphDestroy(p->graph);
    if (p->chunk_counts) cudaFree(p->chunk_counts);
    if (p->pinned_poses) cudaFreeHost(p->pinned_poses);
    if (p->done) cudaEventDestroy(p->done);
    if (p->cap_stream) cudaStreamDestroy(p->cap_stream);
    delete p;
}

extern "C" nif_status nif_sync_status(nif_handle* h, void* stream) {
    if (!h) return NIF_ERR_ARG;
    NIF_CK(h, cudaStreamSynchronize((cudaStream_t)stream));
    int st = 0;
    NIF_CK(h, cudaMemcpy(&st, h->d_status, sizeof(int), cudaMemcpyDeviceToHost));
    if (st != 0) {
        NIF_CK(h, cudaMemset(h->d_status, 0, sizeof(int)));
        return nif_fail(h, (nif_status)st, "device-side error latched by a kernel");
    }
    return NIF_OK;
}
