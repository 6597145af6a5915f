// nif_internal.cuh -- shared internals of the CUDA library (handle, device
// math of the deformation, launch helpers). Not part of the public ABI.
#pragma once

#include <cuda_runtime.h>
#include <cuda_fp16.h>
#include <cuda_bf16.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/nif.h"

#define NIF_MAX_LEVELS 32
#define NIF_MAX_LAYERS 10
#define NIF_OUT 16            // stored output rows (occ, dist, n3, albedo3, M material, pad)
#define NIF_KBEND 0.75f       // bend curvature per unit bend parameter
#define NIF_EPS_DIST 1e-2f    // log-distance epsilon (voxel units)

// ---------------------------------------------------------------------------
// Bounds build. Compiled with -DNIF_BOUNDS=1, NIF_IN(i, n) checks 0 <= i < n
// at the index computations that use it (the grid cell of every encoder
// gather and scatter, label triangles, the rest-space point order, the
// per-ray segment rows); a failed check adds one to this translation unit's
// device word and the caller redirects or skips the access, so nothing
// traps. nif_bounds_check() (include/nif.h) sums and clears the words of
// every translation unit. In the normal build NIF_IN is the constant true
// and compiles away.
// ---------------------------------------------------------------------------
#if defined(NIF_BOUNDS) && NIF_BOUNDS
int nif_bounds_register(unsigned long long (*take)());
namespace {
__device__ unsigned long long nif_bounds_word;
__device__ __forceinline__ bool nif_in_bounds(long long i, long long n) {
    if (i >= 0 && i < n) return true;
    atomicAdd(&nif_bounds_word, 1ull);
    return false;
}
unsigned long long nif_bounds_take() {
    unsigned long long v = 0, z = 0;
    if (cudaMemcpyFromSymbol(&v, nif_bounds_word, sizeof v) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    cudaMemcpyToSymbol(nif_bounds_word, &z, sizeof z);
    return v;
}
const int nif_bounds_registered = nif_bounds_register(&nif_bounds_take);
}  // namespace
#define NIF_IN(i, n) nif_in_bounds((long long)(i), (long long)(n))
#else
#define NIF_IN(i, n) true
#endif

// ---------------------------------------------------------------------------
// Encoding constants passed by value to kernels.
// ---------------------------------------------------------------------------
struct GridInfo {
    int L, Fd, P, F;          // levels, features, gamma terms (1+2F), bands
    uint32_t T;               // entries per level (power of two)
    uint32_t dense_mask;      // bit l set when level l is dense ((N_l+1)^3 <= T)
    int res[NIF_MAX_LEVELS];  // N_l
};

// Learned deformation field of the instances (see the device math below).
#define NIF_FIELD_MAX_G 33
#define NIF_FIELD_MAX_LIPSCHITZ 0.9f
struct FieldView {
    const float4* d = nullptr;   // [n][G^3] (delta, 0); nullptr: no field
    int G = 0;
    int n = 0;                   // instances that have a field
};

// Octree over the occupied voxels (Morton order). Global node numbering:
// leaves [0, n_leaves), then each internal level in turn; internal node i
// (global index >= n_leaves) has children [child_begin, child_begin + count).
struct TreeView {
    int n_leaves;             // occupied voxels
    int n_nodes;              // leaves + internal nodes
    int top_begin, top_count; // nodes the traversal starts from
    const int2* child;        // [n_nodes - n_leaves]: (begin, count)
    const uint32_t* leaf_vox; // [n_leaves] rest voxel id of each leaf
};

// Dynamic loss scaling state (device): gradients of the 16-bit training path
// are computed for S * loss; Adam unscales them, or skips the step when any
// is not finite.
struct NifLossScale {
    float scale;      // S
    int clean;        // consecutive finite steps since the last change of S
    int overflow;     // set by the gradient check of the current step
    int skipped;      // steps skipped so far
    double b1t, b2t;  // beta1^t, beta2^t over the t steps taken
    float c1, c2;     // Adam's bias corrections for the next step: 1 / (1 - beta^(t+1))
};

struct nif_handle {
    nif_config cfg{};
    int N = 0, L = 0, Fd = 2, P = 0, in_dim = 0, W = 0, H = 0, n_layers = 0;
    bool concat = false;                // Eq. 1 read as [gamma, phi] (NIF_FLAG_CONCAT_ENCODING)
    int point_w = 0;                    // features of one end point: P*L*F_d, or 3P + L*F_d concatenated
    uint32_t T = 0;
    GridInfo grid{};

    // mesh (device copy)
    float* d_verts = nullptr;
    int* d_tris = nullptr;
    float4* d_tri_geo = nullptr;        // per triangle A, B - A, C - A in 3 float4 (w of the third unused)
    float* d_alb = nullptr;
    uint8_t* d_mat = nullptr;
    int n_verts = 0, n_tris = 0;

    // voxels
    uint8_t* d_occ = nullptr;           // [N^3]
    uint32_t* d_tri_ptr = nullptr;      // [N^3 + 1]
    int32_t* d_tri_idx = nullptr;       // [n_pairs]
    int64_t n_pairs = 0;

    // octree topology
    int n_leaves = 0, n_nodes = 0, top_begin = 0, top_count = 0;
    std::vector<int> level_begin, level_count;   // internal levels, bottom-up
    int2* d_child = nullptr;
    uint32_t* d_leaf_vox = nullptr;             // [n_leaves]
    uint32_t* d_leaf_lat = nullptr;             // [n_leaves] packed (i,j,k) 10 bits each

    // per-instance geometry (grown on demand)
    int inst_cap = 0;
    float* d_corners = nullptr;   // [inst][n_leaves][24]
    float4* d_aabb = nullptr;     // [inst][n_nodes][2] (lo, hi)
    float4* d_pose = nullptr;     // [inst] (kappa, twist, taper, 0)

    // learned deformation field (nif_set_field): per instance G^3 rest-space
    // displacements, [field_n][G^3] (delta, 0); its Adam moments in the same
    // layout, its gradient [field_n][G^3][3], a device word for its Lipschitz
    // bound; target poses of nif_field_step
    float4* d_field = nullptr;
    float4* d_field_m = nullptr;
    float4* d_field_v = nullptr;
    float* d_field_g = nullptr;
    float* d_field_lip = nullptr;
    int field_G = 0, field_n = 0;
    long field_step = 0;
    float4* d_pose_t = nullptr;         // [inst_cap_t] (kappa, twist, taper, 0) of target poses
    int inst_cap_t = 0;

    // parameters: one FP32 buffer [tables | layer 0 .. layer H | s(8)]
    size_t n_params = 0, off_tables = 0, off_s = 0;
    size_t off_layer[NIF_MAX_LAYERS + 1] = {0};
    int lay_out[NIF_MAX_LAYERS] = {0}, lay_in[NIF_MAX_LAYERS] = {0};
    float* d_params = nullptr;
    float* d_grad = nullptr;
    float* d_m = nullptr;
    float* d_v = nullptr;
    __half* d_tables_h = nullptr;       // FP16 copy of the tables
    __nv_bfloat16* d_w_bf16 = nullptr;  // BF16 copy of the weights (layers back to back)
    __half* d_w_f16 = nullptr;          // FP16 copy of the weights
    __nv_bfloat16* d_wt_bf16 = nullptr; // BF16 copy of the transposed weights (layer l: [in_l][out_l])
    __half* d_wt_f16 = nullptr;         // FP16 copy of the transposed weights
    NifLossScale* d_ls = nullptr;       // dynamic loss scale of the mixed-precision training path
    bool lowp_dirty = true;
    // split-TF32 copies of the weights for the FP32 tensor-core MLP: layer l
    // at x3_fwd[l] as [hi; lo] x [out_l][in_l] and at x3_bwd[l] transposed,
    // [hi; lo] x [x3_npad[l]][out_l] (rows in_l .. x3_npad[l] zero)
    float* d_w_x3 = nullptr;
    size_t x3_fwd[NIF_MAX_LAYERS] = {0}, x3_bwd[NIF_MAX_LAYERS] = {0};
    int x3_npad[NIF_MAX_LAYERS] = {0};
    bool x3_dirty = true;
    long adam_step = 0;

    // a second stream for work of a training step that can overlap the main
    // stream's (the layer-0 weight gradient beside the encoding backward);
    // it always forks from and joins back into the caller's stream
    cudaStream_t aux = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    // a third stream for nif_train_steps' next batch, and its ordering events
    cudaStream_t aux2 = nullptr;
    cudaEvent_t ev_batch = nullptr, ev_step = nullptr;
    // nif_train_steps[_rays] run their steps on `hi` (the device's greatest
    // stream priority; the weight-gradient stream `aux` too), forked from and
    // joined back into the caller's stream, so that the next batch on `aux2`
    // (the least priority) takes the SMs the step leaves free
    cudaStream_t hi = nullptr, aux_hi = nullptr;
    cudaEvent_t ev_hi_fork = nullptr, ev_hi_join = nullptr;
    double* h_loss = nullptr;           // pinned: per-step loss parts of nif_train_steps_rays
    int h_loss_steps = 0;

    // device status word + scratch
    int* d_status = nullptr;            // [0] latched status; [2..3] 64-bit wait bound (ns, 0 = 1 s)
    double* d_lossacc = nullptr;        // [16] loss accumulators
    int* d_count = nullptr;             // [4] counters
    uint32_t* d_next = nullptr;         // [4] work counters: [0] rays of the persistent traversal,
                                        // [1] tasks of the encoding backward
    int* h_pinned = nullptr;            // pinned host word(s)

    // grown scratch buffers (query / train)
    struct Buf { void* p = nullptr; size_t bytes = 0; };
    Buf b_counts, b_offsets, b_segs, b_lin, b_feat, b_out, b_acts, b_dout, b_dx, b_labels,
        b_scan, b_rays, b_inst, b_feat2, b_temp, b_dys, b_dup, b_pts, b_lattice, b_sort, b_lin_t,
        b_feat_alt;                     // the other step's FP32 features while its weight gradients run late
    // NIF_KNOB_DETERMINISTIC: gradients summed in an order-free way. b_fix holds
    // the table gradient as 64-bit fixed point ([L][T][F_d] words, zero between
    // calls) followed by two 32-bit words (max |dL/dfeature| bits, scale exponent);
    // b_parts the weight-gradient partial sums of each row range; b_lparts the
    // loss partial sums of each block
    bool det = false;
    Buf b_fix, b_parts, b_lparts;
    // NIF_KNOB_FAIL_ALLOC: the n-th scratch allocation from the knob's setting
    // fails as an out-of-memory cudaMalloc would (host-side fault injection)
    int fail_alloc = 0;
    // FP32 steps with the weight update deferred (NIF_KNOB_DEFER_WEIGHTS): the
    // weights' Adam runs on the second stream after the weight gradients and
    // records ev_wupd; the next step's MLP forward waits for it
    cudaEvent_t ev_wupd = nullptr;
    cudaEvent_t ev_dw[2] = {nullptr, nullptr};   // weight gradients of the last step on batch set k done
    bool wupd_pending = false;
    int feat_flip = 0;
    // set by the training pipeline while the next batch is built beside a
    // step: the step's persistent MLP forward then leaves SMs to that batch
    bool batch_beside = false;
    // the distinct end points of the last segment encoding (in b_dup, b_pts,
    // b_sort; sorted: in rest-space order), which the backward of the same
    // segments in a training step takes instead of listing them again
    struct PointList {
        const nif_linseg* lin = nullptr;
        const uint32_t* n_dev = nullptr;
        int64_t n_max = 0;
        const uint32_t *pts = nullptr, *n_pts = nullptr, *dupf = nullptr;
        bool sorted = false;
    } enc_points;
    int* d_vox_leaf = nullptr;          // [N^3] octree leaf of each voxel, -1 when empty (exit-face walk)
    // the second set of training-batch buffers of nif_train_steps (the next
    // step's batch is built into it while the current step trains)
    Buf alt_counts, alt_offsets, alt_temp, alt_segs, alt_scan, alt_rays, alt_inst, alt_lin, alt_labels, alt_dup,
        alt_pts, alt_sort;
    PointList alt_enc_points;
    double query_seg_per_ray = 0.0;     // segments per ray of the last counted traversal (temp capacity hint)
    // nif_query without host synchronisation: its segment capacity comes from
    // the segments per ray of earlier queries, whose totals are read back
    // asynchronously (pinned word + event), or q_init before the first
    double q_hint = 0.0, q_init = 8.0;
    uint32_t* h_qtotal = nullptr;       // pinned: unclamped total of the last query
    cudaEvent_t ev_qtotal = nullptr;
    bool q_pending = false;
    int q_rays = 0;
    uint32_t* d_chunk_counts = nullptr; // per-chunk segment counts of nif_query
    int chunk_counts_cap = 0;
    // pose uploads of more instances than a kernel argument holds
    float4* h_pose_pinned = nullptr;
    int pose_pinned_cap = 0;
    cudaEvent_t ev_pose = nullptr;
    bool pose_pending = false;
    double seg_scratch_scale = 1.0;     // NIF_KNOB_SEG_SCRATCH: scale of the single-traversal segment scratch

    // launch knobs chosen by the autotuner (nif_query_plan_create)
    struct Tune {
        int trav_warps = 4;             // warps per traversal block
        int enc_threads = 256;          // encoding block size
        int enc_blocks_per_sm = 16;     // encoding grid cap per SM (grid-stride beyond)
        int64_t tc_chunk = 1 << 20;     // rows per encode + tensor-core MLP chunk
        int step_bwd_ctas = 0;          // NIF_KNOB_STEP_BWD_CTAS: the FP32 step's encoding backward CTAs beside
                                        // the weight gradients (0: seven eighths of the SMs; -1: every SM)
        int bwd_smem_rows = 512;        // encoding backward: dense coarse levels of at most this many rows
                                        // go to shared memory (measured: larger ones reduce faster in L2)
        int batch_at = 0;               // FP32 steps of nif_train_steps: the next batch starts at 0 the step's
                                        // start, 1 after the encoding forward, 2 after the MLP forward, 3 after
                                        // the MLP backward (NIF_KNOB_BATCH_AT; measured: 0 is ~0.01 ms faster
                                        // than 1 on the 64^3 step, 2 and 3 are 0.1-0.2 ms slower)
        int fp32_fused = 1;             // NIF_KNOB_FP32_FUSED: the FP32 forward in one launch (training steps,
                                        // nif_mlp_forward)
        int query_fp32_fused = 1;       // the same for FP32 queries (set by the knob, timed by plan autotuning)
        int step_fwd_ctas = 0;          // NIF_KNOB_STEP_FWD_CTAS: the step's MLP forward CTAs beside the next
                                        // batch (0: FP32 three quarters of the SMs, tile-balanced, 16-bit
                                        // every SM; -1: every SM)
        int defer_wupd = 1;             // NIF_KNOB_DEFER_WEIGHTS: FP32 steps update the weights beside the next step
        int step_prio = 0;              // NIF_KNOB_STEP_PRIORITY: pipelined steps on the high-priority streams
        int query_fused = 1;            // NIF_KNOB_QUERY_FUSED: 16-bit queries encode into the tensor-core
                                        // MLP's shared-memory ring (one launch) instead of two kernels
        int bwd_split = 0;              // NIF_KNOB_BWD_SPLIT: level halves per task of the run-length backward
                                        // (0: 2 when L >= 16, else 1)
        int order_bits = 7;             // NIF_KNOB_ORDER_BITS: the rest-space point order sorts by the Morton
                                        // code of a 2^b-per-axis grid (measured on the 64^3 steps: FP32 2.90 ms
                                        // at 6, 2.79 at 7, 2.85 at 8; BF16 mixed 2.35, 2.22, 2.28; the
                                        // 64-instance batch 41.0-42.6 ms at 5-8, flat)
    } tune;

    // CUDA graphs of live query plans hold the scratch and per-instance
    // buffers by address: while any plan exists, a buffer that has to grow is
    // replaced and the old allocation kept here until the last plan is gone
    int n_plans = 0;
    std::vector<void*> graveyard;

    std::string err;
    int num_sms = 0;
    double seg_per_ray = 0.0;           // measured segments per sampled training ray

    // per-kernel timing (CUDA events on the launching stream), off by default
    struct ProfRec { const char* name; cudaEvent_t a, b; };
    bool prof = false;
    std::string prof_filter;            // comma-separated stage names, or empty for all
    std::vector<ProfRec> prof_recs;
    std::vector<cudaEvent_t> prof_pool;
    size_t prof_used = 0;
    std::vector<std::pair<std::string, std::pair<double, long>>> prof_sum;
};

// Launch counter of every kernel this library enqueues (diagnostics).
void nif_count_launch();

// Scope that brackets the launches of one named stage with CUDA events when
// the handle's profiling is on.
struct NifProf {
    nif_handle* h;
    cudaStream_t s;
    size_t rec = (size_t)-1;
    NifProf(nif_handle* h_, const char* name, cudaStream_t s_);
    ~NifProf();
};

// ---------------------------------------------------------------------------
// Host helpers
// ---------------------------------------------------------------------------
nif_status nif_fail(nif_handle* h, nif_status st, const std::string& msg);
nif_status nif_cuda_fail(nif_handle* h, cudaError_t e, const char* what);
nif_status nif_grow(nif_handle* h, nif_handle::Buf& b, size_t bytes);
// frees `p` now, or keeps it until the last query plan of the handle is destroyed
void nif_retire(nif_handle* h, void* p);
// frees the retired buffers (no plan may be alive)
void nif_free_retired(nif_handle* h);
nif_status nif_ensure_instances(nif_handle* h, int n_inst);
nif_status nif_upload_poses(nif_handle* h, const nif_pose* poses, int n_inst, cudaStream_t s);
nif_status nif_refresh_lowp(nif_handle* h, cudaStream_t s);
// argument checks shared by the entry points that take poses and rays
nif_status nif_check_inst(nif_handle* h, const nif_pose* poses, int n_inst, const int* inst_off, int n_rays);
// synchronises s, then returns (and clears) the device status word
nif_status nif_check_status(nif_handle* h, cudaStream_t s);
// loss scale back to its initial value (FP16 handles 2^15, others 1), counters cleared (blocking)
nif_status reset_loss_scale(nif_handle* h);

#define NIF_CK(h, call)                                                   \
    do {                                                                  \
        cudaError_t e_ = (call);                                          \
        if (e_ != cudaSuccess) return nif_cuda_fail((h), e_, #call);      \
    } while (0)

#define NIF_CK_LAUNCH(h)                                                  \
    do {                                                                  \
        nif_count_launch();                                               \
        cudaError_t e_ = cudaGetLastError();                              \
        if (e_ != cudaSuccess) return nif_cuda_fail((h), e_, "launch");   \
    } while (0)

static inline unsigned nif_blocks(int64_t n, int threads) {
    int64_t b = (n + threads - 1) / threads;
    return (unsigned)(b < 1 ? 1 : b);
}

// ---------------------------------------------------------------------------
// Kernel launchers (defined in the k_*.cu files)
// ---------------------------------------------------------------------------
nif_status nif_voxelize_run(nif_handle* h);
nif_status nif_refit_run(nif_handle* h, int n_inst, cudaStream_t s);
nif_status nif_seg_count_run(nif_handle* h, const nif_ray* rays, const int* inst_off, int n_inst,
                             int n_rays, uint32_t* counts, cudaStream_t s);
nif_status nif_scan_run(nif_handle* h, const uint32_t* in, uint32_t* out, int n, cudaStream_t s);
nif_status nif_seg_temp_run(nif_handle* h, const nif_ray* rays, const int* inst_off, int n_inst, int n_rays,
                            uint32_t* counts, nif_segment* temp, int64_t temp_cap, uint32_t* cursor,
                            cudaStream_t s);
nif_status nif_seg_scatter_run(nif_handle* h, const nif_segment* temp, const uint32_t* n_temp,
                               int64_t n_temp_max, const uint32_t* offsets, uint32_t* fill, int n_rays,
                               nif_segment* segs, int64_t cap, cudaStream_t s);
nif_status nif_seg_emit_run(nif_handle* h, const nif_ray* rays, const int* inst_off, int n_inst,
                            int n_rays, const uint32_t* offsets, nif_segment* segs, int64_t cap,
                            cudaStream_t s);
nif_status nif_linearize_run(nif_handle* h, const nif_ray* rays, const int* inst_off, int n_inst,
                             const nif_segment* segs, const uint32_t* n_segs_dev, int64_t n_max,
                             nif_linseg* lin, cudaStream_t s);
// linearization by explicit device poses and field (no field: f.d == nullptr)
nif_status nif_linearize_with_run(nif_handle* h, const nif_ray* rays, const int* inst_off, int n_inst,
                                  const float4* poses_dev, FieldView f, const nif_segment* segs,
                                  const uint32_t* n_segs_dev, int64_t n_max, nif_linseg* lin, cudaStream_t s);
// gradient of sum(dL/dp . p) with respect to the field: dfield [field_n][G^3][3] (accumulated)
nif_status nif_field_grad_run(nif_handle* h, const nif_segment* segs, const nif_linseg* lin, const float* dp,
                              const uint32_t* n_dev, int64_t n, const int* inst_off, int n_inst, float* dfield,
                              cudaStream_t s);
// Adam on the field from h->d_field_g (then cleared), then the field scaled
// back to the Lipschitz bound NIF_FIELD_MAX_LIPSCHITZ where a step passed it
nif_status nif_field_adam_run(nif_handle* h, float lr, cudaStream_t s);
// frees the field's buffers (nif_destroy)
void nif_field_free(nif_handle* h);
nif_status nif_encode_points_run(nif_handle* h, const float* pts, int64_t n, void* feats,
                                 int out_dtype, int32_t* rows, cudaStream_t s);
// reuse_points: the list of distinct end points that nif_encode_points_prepare
// (or an earlier encoding) made for the same lin / n_dev / n_max, on this
// stream, is taken as it is
// dedup: encode only the distinct end points (a device-side list prepared
// per call); off, every (segment, end point) is encoded without preparation
nif_status nif_encode_segments_run(nif_handle* h, const nif_linseg* lin, const uint32_t* n_dev,
                                   int64_t n_max, void* feats, int out_dtype, int table_dtype,
                                   cudaStream_t s, bool reuse_points = false, bool dedup = true);
// the distinct end points of a training batch, built with the batch (on its
// stream) for the forward and backward encodings of the step that trains on it
nif_status nif_encode_points_prepare(nif_handle* h, const nif_linseg* lin, const uint32_t* n_dev,
                                     int64_t n_max, int table_dtype, cudaStream_t s);
nif_status nif_encode_points_bwd_run(nif_handle* h, const float* pts, int64_t n, const float* dfeats,
                                     float* dtables, float* dpts, cudaStream_t s);
// reuse_points: the segment encoding just before, on the same stream, read the
// same lin / n_dev / n_max; its list of distinct end points is taken as it is.
// ctas > 0 caps the persistent run-length kernel's CTAs (0: one per SM)
nif_status nif_encode_segments_bwd_run(nif_handle* h, const nif_linseg* lin, const uint32_t* n_dev,
                                       int64_t n_max, const float* dfeats, float* dtables,
                                       cudaStream_t s, bool reuse_points = false, int ctas = 0);
nif_status nif_encode_segments_dp_run(nif_handle* h, const nif_linseg* lin, const uint32_t* n_dev, int64_t n,
                                      const float* dfeats, float* dp, cudaStream_t s);
nif_status nif_pose_grad_run(nif_handle* h, const nif_segment* segs, const nif_linseg* lin, const float* dp,
                             const uint32_t* n_dev, int64_t n, const int* inst_off, int n_inst, float* dposes,
                             cudaStream_t s);
// FP32 MLP on the tensor cores (split TF32, k_mlp_x3.cu); acts [H][n_max][W]
// ctas > 0 caps the one-launch forward's persistent CTAs. query: the hidden
// activations are not needed (acts is then scratch for the per-layer launches
// only) and the one-launch choice is tune.query_fp32_fused, not fp32_fused
nif_status nif_mlp_fwd_fp32_run(nif_handle* h, const float* x, const uint32_t* n_dev, int64_t n_max,
                                float* out, float* acts, cudaStream_t s, int ctas = 0, bool query = false);
// want_dw: add dL/dW into the gradient buffer (off for an input gradient only);
// with `aux`, the weight gradients run there (forked from s once every dY_l is
// ready; the caller joins with h->ev_join before reading gradients)
nif_status nif_mlp_bwd_fp32_run(nif_handle* h, const float* x, const uint32_t* n_dev, int64_t n_max,
                                const float* acts, const float* dout, float* dx, cudaStream_t s,
                                bool want_dw = true, cudaStream_t aux = nullptr);
// exit-face walk of the deformed grid (k_segment.cu); mode 0 counts, 1 emits
// into the rows of `offsets`, 2 counts 1 per ray whose first BVH query finds a hull
nif_status nif_seg_walk_run(nif_handle* h, const nif_ray* rays, const int* inst_off, int n_inst, int n_rays,
                            uint32_t* counts, const uint32_t* offsets, nif_segment* segs, int64_t cap, int mode,
                            cudaStream_t s);
nif_status nif_x3_alloc(nif_handle* h);
nif_status nif_refresh_x3(nif_handle* h, cudaStream_t s);
// The query path's encoding and tensor-core MLP in one persistent launch
// (k_mlp_enc.cu): features never reach global memory. Applies to BF16/FP16
// handles with L in {4, 8, 16}, F_d = 2, W in {32, 64} (nif_mlp_enc_fusable).
bool nif_mlp_enc_fusable(const nif_handle* h);
nif_status nif_mlp_enc_tc_run(nif_handle* h, const nif_linseg* lin, const uint32_t* n_dev, int64_t n_max, float* out,
                              cudaStream_t s);
nif_status nif_mlp_fwd_tc_run(nif_handle* h, const void* x, int dtype, const uint32_t* n_dev,
                              int64_t n_max, float* out, cudaStream_t s);
// acts_out (nullable): 16-bit hidden activations, layer l row r at (l * acts_rows + r) * acts_ld
// (ctas > 0 caps its persistent CTAs)
nif_status nif_mlp_fwd_tc_acts_run(nif_handle* h, const void* x, int dtype, const uint32_t* n_dev, int64_t n_max,
                                   float* out, uint16_t* acts_out, int64_t acts_rows, int acts_ld, cudaStream_t s,
                                   int ctas = 0);
// 16-bit backward in the handle's precision: dY_l (scaled by the loss scale) into
// dys [H+1][n_pad][ld], dx [n][in_dim] FP32 (scaled)
nif_status nif_mlp_bwd_tc_run(nif_handle* h, const float* dout, const uint16_t* acts, const uint32_t* n_dev,
                              int64_t n_max, int64_t n_pad, int ld, uint16_t* dys, float* dx, cudaStream_t s);
// dW_l += dY_l^T X_l into the gradient buffer (FP32, scaled)
nif_status nif_mlp_dw_tc_run(nif_handle* h, const void* x16, const uint16_t* acts, const uint16_t* dys,
                             const uint32_t* n_dev, int64_t n_max, int64_t n_pad, int ld, cudaStream_t s);
nif_status nif_grad_check_run(nif_handle* h, cudaStream_t s);
nif_status nif_shadow_rays_run(nif_handle* h, const nif_ray* rays, const nif_hit* hits, int n, const float* light,
                               float eps, float tmax, nif_ray* out, cudaStream_t s);
// v[0..n) /= the loss scale (device)
nif_status nif_unscale_run(nif_handle* h, float* v, int n, cudaStream_t s);
nif_status nif_adam_scaled_run(nif_handle* h, float lr_grid, float lr_mlp, cudaStream_t s);
nif_status nif_labels_count_hits(nif_handle* h, const nif_label* labels, int64_t n, cudaStream_t s);
// n_hit (device int, default the handle's first counter word): the count of
// labelled hits, written by nif_labels_run and read by nif_loss_run
// the labels' per-triangle records (d_tri_geo) from d_verts and d_tris
nif_status nif_tri_geo_run(nif_handle* h, cudaStream_t s);
nif_status nif_labels_run(nif_handle* h, const nif_segment* segs, const nif_linseg* lin,
                          const uint32_t* n_dev, int64_t n_max, nif_label* labels, cudaStream_t s,
                          int* n_hit = nullptr);
// want_ds: add dL/ds into the gradient buffer (off for a gradient with respect to the poses only)
nif_status nif_loss_run(nif_handle* h, const float* out, const nif_label* labels,
                        const nif_linseg* lin, const uint32_t* n_dev, int64_t n_max, float* dout,
                        cudaStream_t s, bool want_ds = true, const int* n_hit = nullptr);
nif_status nif_adam_run(nif_handle* h, float lr_grid, float lr_mlp, cudaStream_t s);
// grad[e] += sum over y = 0 .. ny-1, in that order, of part[y * cnt + e]
// (the order-fixed reduction of per-range partial sums in deterministic mode)
nif_status nif_sum_parts_run(nif_handle* h, const float* part, int ny, int64_t cnt, float* grad, cudaStream_t s);
// Adam over the tables (on s_tab) and over the weights and log-variances (on
// s_w) as two launches of the same step (one step count, the same bias
// corrections); false from *split when the ranges cannot be split on
// 16-byte boundaries (then nothing is launched)
nif_status nif_adam_split_run(nif_handle* h, float lr_grid, float lr_mlp, cudaStream_t s_tab, cudaStream_t s_w,
                              bool* split);
nif_status nif_reconstruct_run(nif_handle* h, const nif_ray* rays, const int* inst_off, int n_inst,
                               int n_rays, const uint32_t* offsets, const nif_segment* segs,
                               int64_t seg_cap, const nif_linseg* lin, const float* out,
                               nif_hit* hits, unsigned flags, cudaStream_t s, const uint32_t* n_valid = nullptr);
// n rays of each of the streams stream_id .. stream_id + n_streams - 1, stream after stream
nif_status nif_sample_rays_run(nif_handle* h, unsigned long long seed, int stream_id, int n,
                               nif_ray* rays, cudaStream_t s, int n_streams = 1);
nif_status nif_scan_run_with(nif_handle* h, const uint32_t* in, uint32_t* out, int n, uint32_t* bsum,
                             cudaStream_t s);
// counts[c] = clamp(*n_dev - c * chunk, 0, chunk) for c < n_chunks
nif_status nif_chunk_counts_run(nif_handle* h, const uint32_t* n_dev, int64_t chunk, int n_chunks, uint32_t* counts,
                                cudaStream_t s);
// elements per block of the scan: nif_scan_run_with needs a block-sum buffer of
// ceil(n / NIF_SCAN_BLOCK) + 1 words
constexpr int NIF_SCAN_BLOCK = 1024;
// n_out = min(offsets[n_rays], cap), or with whole_rays the largest offsets[r] <= cap
// (only complete rows); latch: an overflow latches NIF_ERR_CAPACITY (a
// truncated query), otherwise it is the normal end of a training batch
nif_status nif_clamp_count_run(nif_handle* h, const uint32_t* offsets, int n_rays, int64_t cap,
                               uint32_t* n_out, bool latch, cudaStream_t s, bool whole_rays = false);
// emit pass that runs only if a temp pass overflowed (*temp_cursor > temp_cap)
nif_status nif_seg_emit_if_overflow_run(nif_handle* h, const nif_ray* rays, const int* inst_off, int n_inst,
                                        int n_rays, const uint32_t* offsets, nif_segment* segs, int64_t cap,
                                        uint32_t* temp_cursor, int64_t temp_cap, cudaStream_t s);

// ---------------------------------------------------------------------------
// Device math: deformation D = Bend o Twist o Taper about c = (0.5,0.5,0.5)
// (FP32; kappa = NIF_KBEND * bend). Written without 1/kappa so that kappa -> 0
// is the identity.
// ---------------------------------------------------------------------------
__device__ __forceinline__ float nif_sinc(float u) {
    return fabsf(u) < 1e-4f ? 1.0f - u * u * (1.0f / 6.0f) : sinf(u) / u;
}
__device__ __forceinline__ float nif_atanc(float u) {
    return fabsf(u) < 1e-4f ? 1.0f - u * u * (1.0f / 3.0f) : atanf(u) / u;
}

// pose: (kappa, twist, taper)
__device__ __forceinline__ float3 nif_deform(float3 x, float4 pose) {
    float px = x.x - 0.5f, py = x.y - 0.5f, pz = x.z - 0.5f;
    float s = 1.0f + pose.z * pz;                  // taper
    float ax = s * px, ay = s * py;
    float sa, ca;
    sincosf(pose.y * pz, &sa, &ca);                // twist
    float bx = ca * ax - sa * ay, by = sa * ax + ca * ay;
    float be = pose.x * pz;                        // bend
    float sb, cb;
    sincosf(be, &sb, &cb);
    float hb = 0.5f * be;
    float X = bx * cb + pz * sinf(hb) * nif_sinc(hb);
    float Z = pz * nif_sinc(be) - bx * sb;
    return make_float3(X + 0.5f, by + 0.5f, Z + 0.5f);
}

__device__ __forceinline__ float3 nif_inverse(float3 y, float4 pose) {
    float X = y.x - 0.5f, Y = y.y - 0.5f, Z = y.z - 0.5f;
    float k = pose.x;
    float g = 1.0f - k * X, hz = k * Z;            // inverse bend
    float r = sqrtf(g * g + hz * hz);
    float x = (2.0f * X - k * (X * X + Z * Z)) / (1.0f + r);
    float z = (Z / g) * nif_atanc(hz / g);
    float sa, ca;                                  // inverse twist
    sincosf(pose.y * z, &sa, &ca);
    float tx = ca * x + sa * Y, ty = -sa * x + ca * Y;
    float s = 1.0f + pose.z * z;                   // inverse taper
    return make_float3(tx / s + 0.5f, ty / s + 0.5f, z + 0.5f);
}

// Columns of J = dD/dx at the rest point x.
__device__ __forceinline__ void nif_jacobian_cols(float3 x, float4 pose, float3& j0, float3& j1,
                                                  float3& j2) {
    float px = x.x - 0.5f, py = x.y - 0.5f, pz = x.z - 0.5f;
    float s = 1.0f + pose.z * pz;
    float ax = s * px, ay = s * py;
    float sa, ca;
    sincosf(pose.y * pz, &sa, &ca);
    float bx = ca * ax - sa * ay, by = sa * ax + ca * ay;
    float sb, cb;
    sincosf(pose.x * pz, &sb, &cb);
    float m = 1.0f - pose.x * bx;
    // Jt = [[s,0,ta px],[0,s,ta py],[0,0,1]]
    // Jw = [[ca,-sa,-th by],[sa,ca,th bx],[0,0,1]]
    // Jb = [[cb,0,m sb],[0,1,0],[-sb,0,m cb]]
    float th = pose.y, ta = pose.z;
    // T = Jw * Jt
    float T00 = ca * s, T01 = -sa * s, T02 = ca * ta * px - sa * ta * py - th * by;
    float T10 = sa * s, T11 = ca * s, T12 = sa * ta * px + ca * ta * py + th * bx;
    // J = Jb * T, with T row 2 = (0, 0, 1)
    j0 = make_float3(cb * T00, T10, -sb * T00);
    j1 = make_float3(cb * T01, T11, -sb * T01);
    j2 = make_float3(cb * T02 + m * sb, T12, -sb * T02 + m * cb);
}

// Columns of dD/d(kappa, twist, taper) at the rest point x (kappa is the
// curvature; dD/d(bend) = NIF_KBEND * dD/dkappa).
__device__ __forceinline__ void nif_param_jacobian_cols(float3 x, float4 pose, float3& dk, float3& dth,
                                                        float3& dta) {
    float px = x.x - 0.5f, py = x.y - 0.5f, pz = x.z - 0.5f;
    float s = 1.0f + pose.z * pz;
    float ax = s * px, ay = s * py;
    float sa, ca;
    sincosf(pose.y * pz, &sa, &ca);
    float bx = ca * ax - sa * ay, by = sa * ax + ca * ay;
    float be = pose.x * pz;
    float sb, cb;
    sincosf(be, &sb, &cb);
    // bend: d/dkappa at fixed (bx, pz) with h1 = (be sb - 1 + cb)/be^2, h2 = (be cb - sb)/be^2
    float h1, h2;
    if (fabsf(be) < 0.25f) {
        float b2 = be * be;
        h1 = 0.5f - b2 * (1.0f / 8.0f) + b2 * b2 * (1.0f / 144.0f) - b2 * b2 * b2 * (1.0f / 5760.0f);
        h2 = be * (-1.0f / 3.0f + b2 * (1.0f / 30.0f) - b2 * b2 * (1.0f / 840.0f));
    } else {
        h1 = (be * sb - 1.0f + cb) / (be * be);
        h2 = (be * cb - sb) / (be * be);
    }
    dk = make_float3(-bx * pz * sb + pz * pz * h1, 0.f, -bx * pz * cb + pz * pz * h2);
    // twist: d(b)/dtheta = pz (-by, bx, 0), then through the bend Jacobian
    float tx = -pz * by, ty = pz * bx;
    dth = make_float3(cb * tx, ty, -sb * tx);
    // taper: d(a)/dta = pz (px, py, 0), through the twist then the bend
    float ux = pz * px, uy = pz * py;
    float wx = ca * ux - sa * uy, wy = sa * ux + ca * uy;
    dta = make_float3(cb * wx, wy, -sb * wx);
}

// ---------------------------------------------------------------------------
// Learned deformation field (our reading of the paper's future work, Sec. 4):
// per instance a lattice of G^3 rest-space displacements delta (node (i,j,k)
// at (i,j,k)/(G-1), stored [inst][k][j][i] as float4), interpolated
// trilinearly at p clamped to [0,1]^3: u(p). The instance's deformation is
// D(p) = D_pose(p + u(p)); its inverse takes q = D_pose^-1(x) and solves
// p + u(p) = q by Newton's method. The field's Lipschitz bound is kept at
// NIF_FIELD_MAX_LIPSCHITZ or below, so the root is unique and
// |p - p*| <= |p + u(p) - q| / (1 - bound).
// ---------------------------------------------------------------------------

inline FieldView nif_field_view(const nif_handle* h) {
    FieldView f;
    f.d = h->field_G > 0 ? h->d_field : nullptr;
    f.G = h->field_G;
    f.n = h->field_n;
    return f;
}

__device__ __forceinline__ void nif_field_cell(int G, float3 p, int& i, int& j, int& k, float3& t) {
    const float s = (float)(G - 1);
    const float x = fminf(fmaxf(p.x, 0.f), 1.f) * s, y = fminf(fmaxf(p.y, 0.f), 1.f) * s,
                z = fminf(fmaxf(p.z, 0.f), 1.f) * s;
    i = min((int)floorf(x), G - 2);
    j = min((int)floorf(y), G - 2);
    k = min((int)floorf(z), G - 2);
    t = make_float3(x - (float)i, y - (float)j, z - (float)k);
}

// u(p) and, if g != nullptr, the columns g[a] = du/dp_a (zero along a
// coordinate where p lies outside [0,1], where u is constant)
__device__ __forceinline__ float3 nif_field_eval(const FieldView& f, int inst, float3 p, float3* g) {
    const int G = f.G;
    int i, j, k;
    float3 t;
    nif_field_cell(G, p, i, j, k, t);
    const float4* D = f.d + (int64_t)inst * G * G * G;
    float3 u = make_float3(0.f, 0.f, 0.f);
    float3 g0 = u, g1 = u, g2 = u;
#pragma unroll
    for (int c = 0; c < 8; c++) {
        const int a = c & 1, b = (c >> 1) & 1, e = (c >> 2) & 1;
        const float4 v = __ldg(D + ((int64_t)(k + e) * G + (j + b)) * G + (i + a));
        const float fx = a ? t.x : 1.f - t.x, fy = b ? t.y : 1.f - t.y, fz = e ? t.z : 1.f - t.z;
        const float w = fx * fy * fz;
        u.x += w * v.x;
        u.y += w * v.y;
        u.z += w * v.z;
        if (g) {
            const float s = (float)(G - 1);
            const float wx = (a ? s : -s) * fy * fz, wy = (b ? s : -s) * fx * fz, wz = (e ? s : -s) * fx * fy;
            g0.x += wx * v.x; g0.y += wx * v.y; g0.z += wx * v.z;
            g1.x += wy * v.x; g1.y += wy * v.y; g1.z += wy * v.z;
            g2.x += wz * v.x; g2.y += wz * v.y; g2.z += wz * v.z;
        }
    }
    if (g) {
        const float ox = (p.x >= 0.f && p.x <= 1.f) ? 1.f : 0.f, oy = (p.y >= 0.f && p.y <= 1.f) ? 1.f : 0.f,
                    oz = (p.z >= 0.f && p.z <= 1.f) ? 1.f : 0.f;
        g[0] = make_float3(g0.x * ox, g0.y * ox, g0.z * ox);
        g[1] = make_float3(g1.x * oy, g1.y * oy, g1.z * oy);
        g[2] = make_float3(g2.x * oz, g2.y * oz, g2.z * oz);
    }
    return u;
}

// x = A^-1 r for A with columns c0, c1, c2 (Cramer's rule)
__device__ __forceinline__ float3 nif_solve3(float3 c0, float3 c1, float3 c2, float3 r) {
    const float3 x01 = make_float3(c1.y * c2.z - c1.z * c2.y, c1.z * c2.x - c1.x * c2.z, c1.x * c2.y - c1.y * c2.x);
    const float det = c0.x * x01.x + c0.y * x01.y + c0.z * x01.z;
    const float inv = 1.0f / det;
    const float3 a = make_float3(r.y * c2.z - r.z * c2.y, r.z * c2.x - r.x * c2.z, r.x * c2.y - r.y * c2.x);
    const float3 b = make_float3(c1.y * r.z - c1.z * r.y, c1.z * r.x - c1.x * r.z, c1.x * r.y - c1.y * r.x);
    return make_float3((r.x * x01.x + r.y * x01.y + r.z * x01.z) * inv,
                       (c0.x * a.x + c0.y * a.y + c0.z * a.z) * inv,
                       (c0.x * b.x + c0.y * b.y + c0.z * b.z) * inv);
}

// x = A^-T r for A with columns c0, c1, c2: the rows of A^T are c0, c1, c2
__device__ __forceinline__ float3 nif_solve3_t(float3 c0, float3 c1, float3 c2, float3 r) {
    return nif_solve3(make_float3(c0.x, c1.x, c2.x), make_float3(c0.y, c1.y, c2.y), make_float3(c0.z, c1.z, c2.z), r);
}

// p with p + u(p) = q: Newton from one fixed-point step, until the FP32
// residual stops shrinking (at most 12 iterations)
__device__ __forceinline__ float3 nif_field_inverse(const FieldView& f, int inst, float3 q) {
    float3 u = nif_field_eval(f, inst, q, nullptr);
    float3 p = make_float3(q.x - u.x, q.y - u.y, q.z - u.z);
    float prev = 3.0e38f;
    for (int it = 0; it < 12; it++) {
        float3 g[3];
        u = nif_field_eval(f, inst, p, g);
        const float3 F = make_float3(p.x + u.x - q.x, p.y + u.y - q.y, p.z + u.z - q.z);
        const float r = fmaxf(fabsf(F.x), fmaxf(fabsf(F.y), fabsf(F.z)));
        if (r == 0.f || r >= prev) break;
        prev = r;
        const float3 dp = nif_solve3(make_float3(1.f + g[0].x, g[0].y, g[0].z),
                                     make_float3(g[1].x, 1.f + g[1].y, g[1].z),
                                     make_float3(g[2].x, g[2].y, 1.f + g[2].z), F);
        p = make_float3(p.x - dp.x, p.y - dp.y, p.z - dp.z);
    }
    return p;
}

__device__ __forceinline__ float3 nif_cross(float3 a, float3 b) {
    return make_float3(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x);
}

__device__ __forceinline__ void nif_set_status(int* status, int code) {
    atomicCAS(status, 0, code);
}
