/*
 * nif.h -- C ABI of the GB300 (sm_103a) implementation of the voxel
 * deformation-aware neural intersection function (Kao, Makowski, Fujieda,
 * Harada, "Voxel Deformation-Aware Neural Intersection Function", 2026).
 *
 * The method (Sec. 2): geometry is voxelized in a rest space; a
 * parameterized deformation moves the voxels into a deformed space where rays
 * are traced as straight lines (Sec. 2.1). Each ray / occupied-voxel segment
 * is mapped back to rest space by the inverse deformation and approximated by
 * a straight rest segment (local linearization, Sec. 2); its end points are
 * encoded by psi = phi o gamma (positional encoding followed by a
 * multiresolution hash grid, Eq. 1) and an MLP predicts occlusion, distance,
 * normal, albedo and material. Distances are reconstructed along the
 * segmented ray (Sec. 2.2). Training uses task losses combined by learned
 * uncertainty weights (Sec. 2.4).
 *
 * Conventions shared by every entry point
 *  - Every call returns nif_status; no C++ exception crosses this ABI.
 *  - "_dev" pointers are CUDA device pointers owned by the caller; "_host"
 *    pointers are host memory owned by the caller. The library owns only the
 *    memory behind a nif_handle (mesh copy, voxels, parameters, optimizer
 *    state, scratch), allocated in nif_create or grown on demand by a call
 *    that needs more scratch, and freed by nif_destroy.
 *  - `stream` is a cudaStream_t (NULL = legacy default stream). Work is
 *    enqueued on it; a call blocks the host only where its description says
 *    so (it returns a count or a value to host memory).
 *  - A handle is not thread-safe: use one handle per host thread / stream.
 *  - Errors found on the device (segment capacity exceeded, non-finite
 *    loss) are latched in a status word that the next synchronising call
 *    returns; nif_last_error() gives a message for the last failure.
 *  - All floating-point work of the library is FP32 unless stated; the
 *    mixed-precision query path stores hash features in FP16 and runs the
 *    MLP with BF16 or FP16 operands and FP32 accumulation on tensor cores.
 */
#ifndef NIF_H
#define NIF_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct nif_handle nif_handle;

typedef enum {
    NIF_OK = 0,
    NIF_ERR_ARG = -1,       /* invalid argument (null, size, unsupported config) */
    NIF_ERR_CUDA = -2,      /* a CUDA runtime call failed */
    NIF_ERR_OOM = -3,       /* device allocation failed */
    NIF_ERR_CAPACITY = -4,  /* a device-side list overflowed its capacity */
    NIF_ERR_TIMEOUT = -5,   /* a bounded device-side wait gave up */
    NIF_ERR_NAN = -6,       /* non-finite loss or gradient */
    NIF_ERR_STATE = -7      /* call not valid in the handle's state */
} nif_status;

typedef enum { NIF_FP32 = 0, NIF_BF16 = 1, NIF_FP16 = 2 } nif_precision;

/* Sizes of the method. Symbols follow the paper: F frequency bands of the
 * positional encoding, L hash-grid levels (Eq. 1). */
typedef struct {
    int voxel_res;          /* N: rest-space voxel grid N^3 over [0,1]^3; power of two, 2..512 */
    int pe_bands;           /* F: gamma(x) = [x, sin(2^k x), cos(2^k x)]_{k<F} (Eq. 1); 0..8 */
    int levels;             /* L: hash-grid levels (Eq. 1); 1..32 */
    int feats;              /* F_d: features per level; must be 2 */
    int log2_table;         /* T = 2^log2_table entries per level; 4..24 */
    int base_res;           /* N_min: coarsest grid resolution */
    float growth;           /* b: level l has N_l = floor(N_min * b^l) cells per axis */
    int mlp_depth;          /* H hidden ReLU layers; 1..8 */
    int mlp_width;          /* W: hidden width; 16, 32, 64 or 128 */
    int n_materials;        /* M material classes; 1..8 */
    int precision;          /* nif_precision of nif_query's encoding + MLP */
    unsigned flags;         /* NIF_FLAG_* below; 0 = the paper's method */
    unsigned long long seed;/* parameter initialisation and training-sample seed */
} nif_config;

/* Ablation switches (the paper's "Deformed" baseline of Table 1 / Sec. 3.2
 * drops its training and encoding modifications):
 * NIF_FLAG_FIXED_TASK_WEIGHTS  task log-variances s held at 0 (no uncertainty
 *                              weighting, Sec. 2.4): 0.5 L_reg + L_cls;
 * NIF_FLAG_SIGMOID_DISTANCE    distance head sqrt(3) * sigmoid(z) in voxel
 *                              units with a plain squared error, instead of
 *                              the ReLU head and log-space error of Sec. 2.4.
 * (No positional encoding is pe_bands = 0.) */
#define NIF_FLAG_FIXED_TASK_WEIGHTS 1u
#define NIF_FLAG_SIGMOID_DISTANCE 2u

/* NIF_FLAG_MIXED_TRAINING  nif_train_step / nif_train_step_rays run the
 * mixed-precision training path in cfg.precision (BF16 or FP16; W 32 or 64):
 * features encoded from the FP16 table copy into 16-bit rows, tensor-core
 * MLP forward keeping 16-bit activations, loss on the FP32 outputs,
 * tensor-core backward and weight gradients on S * loss with FP32
 * accumulation, FP32 atomic table gradients, FP32 master parameters and
 * Adam on the gradient divided by S. A step whose gradient holds a
 * non-finite value is skipped. S (the loss scale) starts at 2^15 for FP16
 * (halved on a skipped step, doubled after 2000 finite steps) and stays 1
 * for BF16. Sec. 3 of the paper trains with FP16 hash features and FP32
 * master copies; the scaling rule is ours. */
#define NIF_FLAG_MIXED_TRAINING 4u
/* NIF_FLAG_CONCAT_ENCODING: read Eq. 1 (Sec. 2.3) as the concatenation
 * psi(p) = [gamma(p), phi(p)] instead of the default phi(gamma(p)). An end
 * point then gives 3P + L*F_d features: gamma's raw values ordered
 * [term][coordinate] (x, then sin(2^k x), cos(2^k x) for k < F) and the grid
 * features at u = p ordered [level][feature]; a segment's MLP input is
 * [psi(p0), psi(p1)] zero-padded to in_dim = 2(3P + L*F_d) rounded up to a
 * multiple of 16. The point-encoding calls (nif_encode_points and its
 * backward) keep the composed layout and refuse such a handle. */
#define NIF_FLAG_CONCAT_ENCODING 8u
/* NIF_FLAG_BILINEAR_FACES: take each face of a deformed voxel (Sec. 2.1,
 * Sec. 2.2) as the bilinear patch of its four deformed corners instead of
 * the default two triangles split along the diagonal from the face's lowest
 * lattice corner (the paper fixes neither). Segments are then [first, last]
 * hit of the ray line with the six patches, by the same rule as for the
 * triangulated hull. The hit test is not watertight: a ray passing within
 * FP32 rounding of a face edge may miss both faces that share it. The
 * exit-face walk (nif_segments_walk) is defined on the triangulated faces and
 * refuses such a handle. */
#define NIF_FLAG_BILINEAR_FACES 16u

/* Rest-space triangle mesh inside [0,1]^3 (host memory, copied by nif_create). */
typedef struct {
    const float* verts;                 /* [n_verts * 3] */
    int n_verts;
    const int* tris;                    /* [n_tris * 3], outward winding */
    int n_tris;
    const float* tri_albedo;            /* [n_tris * 3] in [0,1], or NULL (0.5) */
    const unsigned char* tri_material;  /* [n_tris] < n_materials, or NULL (0) */
} nif_mesh;

/* Deformation parameters (our reading; the paper names no family):
 * D(x) = c + Bend(Twist(Taper(x - c))), c = (0.5, 0.5, 0.5);
 * Taper s = 1 + taper*z scales (x, y); Twist turns (x, y) by twist*z radians;
 * Bend (Barr 1984) bends the x-z plane with curvature 0.75*bend. */
typedef struct { float bend, twist, taper; } nif_pose;

/* Ray in the deformed space of its instance; d of unit length. 32 bytes. */
typedef struct { float o[3], d[3], tmin, tmax; } nif_ray;

/* Query result of one ray. 32 bytes. hit = 0 means no hit, D = +inf. */
typedef struct {
    float D;              /* distance along the ray to the predicted hit (Sec. 2.2) */
    float n[3];           /* deformed-space unit normal */
    float albedo[3];
    unsigned char hit, material, pad[2];
} nif_hit;

/* One ray / occupied deformed voxel segment (Sec. 2.2). 16 bytes.
 * voxel = i + N*(j + N*k) of the rest voxel; [t0, t1] along the ray. */
typedef struct { uint32_t ray, voxel; float t0, t1; } nif_segment;

/* Linearized rest segment of a nif_segment (Sec. 2). 32 bytes.
 * p0 = D^-1(o + t0 d), p1 = D^-1(o + t1 d); l_def = |x1 - x0|, l_rest = |p1 - p0|. */
typedef struct { float p0[3], p1[3], l_def, l_rest; } nif_linseg;

/* Ground-truth attributes of a linearized segment (Sec. 2). 32 bytes.
 * tpar in [0,1] is the hit parameter along p0 -> p1; normal is the unit
 * geometric normal of the hit triangle in rest space. */
typedef struct {
    float tpar, normal[3], albedo[3];
    unsigned char occ, material, pad[2];
} nif_label;

/* Parameter groups for nif_get_params / nif_set_params (FP32, host memory). */
enum {
    NIF_PARAM_TABLES = 0,   /* [L][T][F_d] hash-grid tables */
    NIF_PARAM_LOGVAR = 1,   /* [5] s_i = log sigma_i^2: distance, normal, albedo, material, occlusion */
    NIF_PARAM_LAYER0 = 16   /* + i: weight of layer i, [out][in] row-major, i = 0..H;
                               layer H is the output layer with 16 rows: 0 occupancy logit,
                               1 distance, 2-4 normal, 5-7 albedo logits, 8.. material logits */
};

/* ------------------------------------------------------------------------ */
/* Lifetime                                                                  */
/* ------------------------------------------------------------------------ */

/* Validates cfg, copies the mesh to the device, voxelizes it in rest space
 * (Sec. 2; triangle/box overlap of voxels dilated by 1e-7) and builds the
 * fixed-topology octree over the occupied voxels used by the per-pose
 * "simple BVH" (Sec. 2.1). Parameters are initialised from cfg->seed
 * (tables U[-1e-4, 1e-4], Kaiming-uniform weights, s = 0). Blocks the host.
 * On failure *out is NULL and nif_last_error(NULL) explains. */
nif_status nif_create(const nif_config* cfg, const nif_mesh* mesh, nif_handle** out);

/* Frees everything the handle owns. NULL is a no-op. Synchronises the device. */
void nif_destroy(nif_handle* h);

/* Message of the last failure on this handle (or of the calling thread's
 * last nif_create when h is NULL). Never NULL; valid until the next call. */
const char* nif_last_error(const nif_handle* h);

/* Size in bytes of a parameter group (see the enum above). */
nif_status nif_param_bytes(const nif_handle* h, int group, size_t* bytes);
/* Copy a parameter group to/from host memory (FP32). Blocks the host.
 * nif_set_params also refreshes the FP16 table copy and resets nothing else. */
nif_status nif_get_params(nif_handle* h, int group, void* dst_host, size_t bytes);
nif_status nif_set_params(nif_handle* h, int group, const void* src_host, size_t bytes);
/* Reset the Adam moments and step counter of the handle. */
nif_status nif_reset_optimizer(nif_handle* h);

/* Checkpoint of the trainable state: a 64-byte header (magic "NIFCKPT1",
 * format version 3, the sizes of the configuration that must match, the Adam
 * step count), then the FP32 parameters, Adam first and second moments, the
 * 40-byte state of the mixed-precision path (loss scale, clean-step and
 * skipped-step counts, the Adam bias-correction products of the steps taken),
 * the learned deformation field's section (a 16-byte header: int32
 * instances, int32 nodes per axis G, int64 Adam step count; then its
 * displacements, first and second moments, [n][G^3] x (x, y, z, 0) FP32
 * each; n = G = 0 without a field), and a CRC-32 (IEEE) of everything before
 * it. nif_checkpoint_bytes gives the size of the handle's current state;
 * save writes into host memory; load checks the header, sizes and CRC
 * (NIF_ERR_ARG on any mismatch, leaving the handle unchanged; NIF_ERR_STATE
 * when the field's shape would change while query plans exist) and restores
 * all of it, adding, resizing or removing the handle's field to match. Both
 * block the host. Sampling is seeded by the caller (step
 * seeds), so a checkpoint plus the next seeds determine the run; with
 * NIF_KNOB_DETERMINISTIC the resumed steps are bit-identical to the
 * uninterrupted ones. */
nif_status nif_checkpoint_bytes(const nif_handle* h, size_t* bytes);
nif_status nif_checkpoint_save(nif_handle* h, void* dst_host, size_t bytes);
nif_status nif_checkpoint_load(nif_handle* h, const void* src_host, size_t bytes);

/* Rest-space voxelization (Sec. 2): occ_host [N^3] (x fastest) gets 1 for
 * occupied voxels. If tri_ptr_host is not NULL it receives [N^3 + 1] offsets
 * and tri_idx_host (capacity `cap`) the ascending triangle ids overlapping
 * each voxel. *n_pairs_host (nullable) gets the total number of pairs.
 * Blocks the host. */
nif_status nif_get_voxels(nif_handle* h, unsigned char* occ_host, int64_t* tri_ptr_host,
                          int32_t* tri_idx_host, int64_t cap, int64_t* n_pairs_host);

/* ------------------------------------------------------------------------ */
/* Stages of the hot path (device buffers, enqueued on `stream`)             */
/* ------------------------------------------------------------------------ */

/* Ray / deformed-voxel segments (Sec. 2.1, Sec. 2.2). Instance i (pose
 * poses_host[i]) owns rays[inst_offsets[i] .. inst_offsets[i+1]);
 * inst_offsets_dev may be NULL when n_inst == 1. For every ray, every
 * occupied voxel whose deformed hull (the hexahedron of its 8 deformed
 * lattice corners, each face split into two triangles along the diagonal
 * from its lowest lattice corner) is hit at least twice gives the segment
 * [max(t_min_hit, tmin), min(t_max_hit, tmax)] when that is non-empty;
 * a ray's segments are sorted by (t0, voxel). Candidates come from a
 * per-pose refit of the octree's boxes.
 * Output: ray_offsets_dev [n_rays + 1] (exclusive scan of the per-ray
 * counts) and segs_dev (capacity seg_cap). *n_segs_host (nullable) receives
 * the total. Blocks the host. segs_dev == NULL only counts. Returns
 * NIF_ERR_CAPACITY (and writes nothing past seg_cap) when the total exceeds
 * seg_cap. */
nif_status nif_segments(nif_handle* h, const nif_pose* poses_host, int n_inst,
                        const nif_ray* rays_dev, const int* inst_offsets_dev, int n_rays,
                        uint32_t* ray_offsets_dev, nif_segment* segs_dev, int64_t seg_cap,
                        int64_t* n_segs_host, void* stream);

/* Segment list by the traversal the paper describes (Sec. 2.1): a BVH query
 * for the first occupied deformed voxel on the ray, then a walk through the
 * exit faces of the deformed voxels (empty ones included), emitting every
 * occupied voxel entered, and a new BVH query past the exit whenever the ray
 * leaves the deformed grid. Same arguments, definition of a segment and
 * outputs as nif_segments (the two lists are equal wherever no hull decision
 * is tied); it exists to compare the paper's traversal with nif_segments'
 * enumeration of every occupied hull. flags: 0, or NIF_WALK_FIRST_HIT to run
 * only the first BVH query (segs_dev must then be NULL; ray_offsets_dev gets
 * the prefix sum of 1 per ray whose query finds a hull) -- the BVH part of
 * the traversal alone, for timing. Uses a device copy of the deformed
 * lattice, (N+1)^3 x 16 bytes per instance, grown on demand. Blocks the host
 * like nif_segments. */
#define NIF_WALK_FIRST_HIT 1u
nif_status nif_segments_walk(nif_handle* h, const nif_pose* poses_host, int n_inst,
                             const nif_ray* rays_dev, const int* inst_offsets_dev, int n_rays,
                             uint32_t* ray_offsets_dev, nif_segment* segs_dev, int64_t seg_cap,
                             int64_t* n_segs_host, unsigned flags, void* stream);

/* Local linearization (Sec. 2): lin_dev[s] from segs_dev[s] for s < n_segs. */
nif_status nif_linearize(nif_handle* h, const nif_pose* poses_host, int n_inst,
                         const nif_ray* rays_dev, const int* inst_offsets_dev, int n_rays,
                         const nif_segment* segs_dev, int64_t n_segs, nif_linseg* lin_dev,
                         void* stream);

/* Hybrid encoding psi(p) = phi(gamma(p)) of rest points (Eq. 1). p is clamped
 * to [0,1]^3; each of the P = 1 + 2F terms of gamma goes through the same
 * hash grid at u = term (x term) or u = (term + 1)/2 (sin, cos terms);
 * level l uses q = fl32(u * N_l), cell i0 = min(floor(q), N_l - 1), the
 * dense index i + j(N_l+1) + k(N_l+1)^2 when (N_l+1)^3 <= T, otherwise the
 * hash (i * 1 ^ j * 2654435761 ^ k * 805459861) mod T, and trilinear weights.
 * feats_dev: [n][P][L][F_d], FP32 (out_dtype NIF_FP32) or BF16/FP16.
 * rows_dev (nullable): [n][P][L] int32 table row of each cell's (0,0,0) corner. */
nif_status nif_encode_points(nif_handle* h, const float* pts_dev, int64_t n, void* feats_dev,
                             int out_dtype, int32_t* rows_dev, void* stream);

/* Encoding of segments: feats_dev [n][2][P][L][F_d] = psi(p0) (+) psi(p1).
 * `table_dtype` NIF_FP32 reads the FP32 tables, NIF_FP16 the FP16 copy. */
nif_status nif_encode_segments(nif_handle* h, const nif_linseg* lin_dev, int64_t n,
                               void* feats_dev, int out_dtype, int table_dtype, void* stream);

/* Backward of nif_encode_points: adds d(sum dfeats * psi)/d(table) into
 * dtables_dev [L][T][F_d] (FP32 atomics; NULL = the handle's own gradient
 * buffer) and, if dpts_dev is not NULL, writes d/dp [n][3] (zero where p was
 * clamped). */
nif_status nif_encode_points_backward(nif_handle* h, const float* pts_dev, int64_t n,
                                      const float* dfeats_dev, float* dtables_dev,
                                      float* dpts_dev, void* stream);

/* Backward of nif_encode_segments (FP32 tables): adds the table gradient of
 * sum(dfeats * features) into dtables_dev [L][T][F_d]. */
nif_status nif_encode_segments_backward(nif_handle* h, const nif_linseg* lin_dev, int64_t n,
                                        const float* dfeats_dev, float* dtables_dev, void* stream);

/* Gradient with respect to the deformation parameters (pose fitting; the
 * paper lists learning deformations as future work). For segments whose
 * deformed end points x0 = o + t0 d, x1 = o + t1 d are held fixed, the rest
 * points are p = D^-1(x; theta); with the tables and weights frozen this adds
 * d(sum dfeats * [psi(p0) (+) psi(p1)])/d(bend, twist, taper) into
 * dposes_dev [n_inst][3] (FP32, accumulated). dfeats_dev [n][in_dim] is the
 * gradient with respect to the MLP input (nif_mlp_backward's dx).
 * dp_dev (nullable, [n][2][3]) receives the intermediate dL/dp0, dL/dp1. */
nif_status nif_pose_gradient(nif_handle* h, const nif_pose* poses_host, int n_inst,
                             const int* inst_offsets_dev, const nif_segment* segs_dev,
                             const nif_linseg* lin_dev, int64_t n, const float* dfeats_dev,
                             float* dposes_dev, float* dp_dev, void* stream);

/* MLP forward (Sec. 2, Fig. 2d): H ReLU layers without bias and a linear
 * output layer; out_dev [n][16] FP32. x_dev [n][in_dim] of x_dtype.
 * precision NIF_FP32 runs FP32 FFMA; NIF_BF16 / NIF_FP16 run tcgen05 tensor
 * cores with FP32 accumulation (x_dtype must then equal precision).
 * acts_dev (nullable, FP32 only): [H][n][W] post-ReLU hidden activations. */
nif_status nif_mlp_forward(nif_handle* h, const void* x_dev, int x_dtype, int64_t n,
                           float* out_dev, int precision, float* acts_dev, void* stream);

/* MLP backward (FP32): given x_dev [n][in_dim], acts_dev from nif_mlp_forward
 * and dout_dev [n][16], adds dL/dW into the handle's gradient buffer and
 * writes dx_dev [n][in_dim] (nullable). */
nif_status nif_mlp_backward(nif_handle* h, const float* x_dev, int64_t n, const float* acts_dev,
                            const float* dout_dev, float* dx_dev, void* stream);

/* MLP backward of the mixed-precision path (tensor cores, cfg.precision BF16
 * or FP16, W 32 or 64, in_dim % 16 == 0). x_dev [n][in_dim] of x_dtype ==
 * cfg.precision (16-byte aligned); the hidden activations are recomputed
 * from x_dev with the current weights. With S the handle's loss scale
 * (nif_loss_scale): dY_H = 16-bit(S * dout_dev), dY_l = 16-bit((dY_{l+1}
 * W_{l+1}) * [act_l > 0]); adds S * dL/dW (FP32 accumulation of the 16-bit
 * products) into the gradient buffer and writes dx_dev [n][in_dim] = FP32
 * dY_0 W_0 (nullable). */
nif_status nif_mlp_backward_lowp(nif_handle* h, const void* x_dev, int x_dtype, int64_t n, const float* dout_dev,
                                 float* dx_dev, void* stream);

/* Loss scale of the mixed-precision path. nif_loss_scale reads S and the
 * number of skipped steps (blocking); nif_set_loss_scale sets S (> 0,
 * blocking). nif_adam_step_scaled: if any weight or table gradient is not
 * finite the step is skipped (gradient cleared, skipped + 1, S halved for
 * FP16 handles); otherwise Adam runs on gradient / S for the tables and
 * weights (the log-variance gradient is taken as it is) with bias
 * correction over the steps taken, and S doubles for FP16 handles after
 * 2000 finite steps in a row. nif_reset_optimizer also resets S. */
nif_status nif_loss_scale(nif_handle* h, float* scale_host, int* skipped_host);
nif_status nif_set_loss_scale(nif_handle* h, float scale);
nif_status nif_adam_step_scaled(nif_handle* h, float lr_grid, float lr_mlp, void* stream);

/* Ground-truth labels (Sec. 2): the straight rest segment p0 -> p1 of lin[s]
 * against the triangles overlapping voxel segs[s].voxel; first hit in
 * [0,1], ties to the smaller triangle id. */
nif_status nif_labels(nif_handle* h, const nif_segment* segs_dev, const nif_linseg* lin_dev,
                      int64_t n, nif_label* labels_dev, void* stream);

/* Task losses and uncertainty weighting (Sec. 2.4) for n segments:
 * distance: ReLU head, mean over hit segments of (log(d+eps) - log(y+eps))^2
 *   with y = tpar * l_rest * N and eps = 1e-2 (voxel units);
 * normal: mean over hits of 1 - cos; albedo: sigmoid, mean L1 over hits and
 * channels; material: cross-entropy over hits; occlusion: BCE with logits
 * over all segments; total = sum_reg (0.5 e^-s L + 0.5 s) + sum_cls
 * (e^-s L + 0.5 s). Writes dout_dev [n][16] (nullable) and adds dL/ds into
 * the gradient buffer; parts_host (nullable, blocks) gets
 * [total, L_dist, L_normal, L_albedo, L_material, L_occ]. */
nif_status nif_loss(nif_handle* h, const float* out_dev, const nif_label* labels_dev,
                    const nif_linseg* lin_dev, int64_t n, float* dout_dev, double* parts_host,
                    void* stream);

/* Gradient buffer (same layout as the parameters) and Adam (beta1 0.9,
 * beta2 0.99, eps 1e-15; learning rate lr_grid for tables and s, lr_mlp
 * for the weights). nif_zero_grad clears it; nif_get_grad / nif_set_grad
 * copy a group out / in (blocking). nif_adam_step clears the gradient. */
nif_status nif_zero_grad(nif_handle* h, void* stream);
nif_status nif_get_grad(nif_handle* h, int group, void* dst_host, size_t bytes);
nif_status nif_set_grad(nif_handle* h, int group, const void* src_host, size_t bytes);
nif_status nif_adam_step(nif_handle* h, float lr_grid, float lr_mlp, void* stream);

/* Per-ray reconstruction (Sec. 2.2): the first segment (in list order) with
 * sigmoid(occupancy) > 0.5 gives D = t0 |d| + t_k, t_k = (dist / N) *
 * l_def / l_rest clamped to [0, l_def]; the normal is J_D^-T n_rest at the
 * predicted rest hit point; albedo = sigmoid, material = argmax.
 * flags & NIF_SHADOW_ONLY fills only hit. */
#define NIF_SHADOW_ONLY 1u
nif_status nif_reconstruct(nif_handle* h, const nif_pose* poses_host, int n_inst,
                           const nif_ray* rays_dev, const int* inst_offsets_dev, int n_rays,
                           const uint32_t* ray_offsets_dev, const nif_segment* segs_dev,
                           const nif_linseg* lin_dev, const float* out_dev, nif_hit* hits_dev,
                           unsigned flags, void* stream);

/* ------------------------------------------------------------------------ */
/* Whole paths                                                               */
/* ------------------------------------------------------------------------ */

/* Query (the inference hot path; the problem of Sec. 2: where does a ray in
 * the deformed space first hit the deformed shape): segments (Sec. 2.1,
 * Sec. 2.2) -> linearization (Sec. 2, Fig. 2c) -> encoding (Sec. 2.3, Eq. 1)
 * -> MLP (cfg.precision; Sec. 2, Fig. 2d) -> reconstruction along the
 * segmented ray (Sec. 2.2), for n_inst deformed instances of the handle's
 * shape. Rays and hits are device buffers of n_rays entries.
 * Does not block the host: every count stays on the device. The segment
 * capacity is 1.5 x the segments per ray of the last earlier query whose
 * total has already come back (read without waiting), or NIF_KNOB_QUERY_SEGS
 * (default 8) per ray before the first; growing scratch synchronises. When a
 * query's segments exceed its capacity, the rays whose segment lists fit are
 * answered, the others report no hit, and NIF_ERR_CAPACITY is latched in the
 * status word (nif_sync_status); the next query sizes for the larger count. */
nif_status nif_query(nif_handle* h, const nif_pose* poses_host, int n_inst,
                     const nif_ray* rays_dev, const int* inst_offsets_dev, int n_rays,
                     nif_hit* hits_dev, unsigned flags, void* stream);

/* One training step on caller-given rays (Sec. 2: ground truth from the rest
 * mesh along the linearized segments; Sec. 2.4: task losses with learned
 * uncertainty weights; FP32, or the mixed-precision path of
 * NIF_FLAG_MIXED_TRAINING): segments of the rays are generated and the
 * batch is the segments of the leading whole rays, in ray order, at most
 * n_segments (a ray whose segments would cross n_segments is left out, so
 * the batch is a deterministic function of the rays and poses). They are
 * labelled, encoded, passed through the MLP, the losses are back-propagated
 * into tables, weights and s, and Adam updates them. loss_host (nullable)
 * receives [total, L_dist, L_normal, L_albedo, L_material, L_occ] and
 * blocks. */
nif_status nif_train_step_rays(nif_handle* h, const nif_pose* poses_host, int n_inst,
                               const nif_ray* rays_dev, const int* inst_offsets_dev, int n_rays,
                               int64_t n_segments, float lr_grid, float lr_mlp, double* loss_host,
                               void* stream);

/* One training step with samples drawn on the device from step_seed (the
 * training of Sec. 2 and Sec. 2.4 over random poses, so that one network
 * serves every deformation): n_poses poses with every parameter U[-1,1] and,
 * per pose, rays whose
 * origins are uniform on the radius-2 sphere about the cube centre aimed at
 * points uniform in [0,1]^3 (counter-based splitmix64 stream), enough rays
 * for n_segments segments. poses_out_host (nullable) receives the poses. */
nif_status nif_train_step(nif_handle* h, int64_t n_segments, int n_poses,
                          unsigned long long step_seed, float lr_grid, float lr_mlp,
                          nif_pose* poses_out_host, double* loss_host, void* stream);

/* n_steps training steps (Sec. 2, Sec. 2.4), exactly what n_steps calls of
 * nif_train_step with the seeds first_seed, first_seed + 1, ... compute, in
 * one call. The batch
 * of a step (sampling, segments, linearization, labels: nothing that depends
 * on the parameters) is built on a second internal stream, into a second set
 * of batch buffers, while the previous step trains, so it costs no time on
 * `stream` after the first. loss_host (nullable): the loss parts of the last
 * step, as nif_train_step gives them. Enqueues on `stream`; the host blocks
 * only to read loss_host and the first time buffers grow. */
nif_status nif_train_steps(nif_handle* h, int n_steps, int64_t n_segments, int n_poses,
                           unsigned long long first_seed, float lr_grid, float lr_mlp, double* loss_host,
                           void* stream);

/* n_steps training steps (Sec. 2, Sec. 2.4) on caller-given rays held in
 * HOST memory: step i trains, as nif_train_step_rays does, on the n_rays rays at
 * rays_host + i * n_rays with the n_inst poses at poses_host + i * n_inst
 * (inst_offsets_dev, a device array shared by all steps, nullable when
 * n_inst == 1). Each step's rays are copied to the device and its batch is
 * built on the second internal stream while the previous step trains
 * (rays_host in pinned memory lets the copy overlap; pageable memory works
 * and serialises). loss_host (nullable): [n_steps][6] loss parts as
 * nif_train_step_rays gives them, each step's read back as the step ends on
 * `stream`; the call then blocks until the last step is done and reports a
 * non-finite loss or a device-side error. Without loss_host it returns once
 * the work is enqueued, and rays_host must stay unchanged until `stream` has
 * completed it. */
nif_status nif_train_steps_rays(nif_handle* h, int n_steps, const nif_pose* poses_host, int n_inst,
                                const nif_ray* rays_host, const int* inst_offsets_dev, int n_rays,
                                int64_t n_segments, float lr_grid, float lr_mlp, double* loss_host,
                                void* stream);

/* Pose fitting (the paper names learned deformations as future work): the
 * gradient of the task loss of Sec. 2.4 with respect to the n_inst
 * deformation parameters, tables, weights and s held fixed, for the
 * segments of rays_dev (the batch rule of nif_train_step_rays; rays for instance i
 * are rays_dev[inst_offsets_dev[i] .. [i+1])): segments -> linearization ->
 * labels -> encoding and MLP in cfg.precision -> loss -> MLP input gradient
 * (FP32, or the tensor-core backward divided by the loss scale) -> the
 * encoding's dL/dp0, dL/dp1 -> through D^-1 as in nif_pose_gradient.
 * Writes dposes_dev [n_inst][3] = dL/d(bend, twist, taper) (FP32); adds
 * nothing to the gradient buffer. loss_host as nif_train_step_rays. */
nif_status nif_pose_step(nif_handle* h, const nif_pose* poses_host, int n_inst, const nif_ray* rays_dev,
                         const int* inst_offsets_dev, int n_rays, int64_t n_segments, float* dposes_dev,
                         double* loss_host, void* stream);

/* ------------------------------------------------------------------------ */
/* Learned deformation fields (the paper, Sec. 4, names learning deformation  */
/* fields jointly with intersection prediction as future work and defines    */
/* none; this parameterisation, its inverse and the fitting objective are     */
/* our reading)                                                                */
/* ------------------------------------------------------------------------ */

/* A field gives each instance i a lattice of G x G x G rest-space
 * displacements delta_i (node (a, b, c) at (a, b, c)/(G-1) of the rest cube),
 * interpolated trilinearly at p clamped to [0,1]^3: u_i(p). With a field the
 * deformation of instance i is D(p) = D_pose_i(p + u_i(p)): a zero field is the
 * parameterised deformation, a zero pose the field alone. Every call that
 * takes poses then uses it: the voxel hulls are the hexahedra of D(lattice
 * corners) (Sec. 2.1), the linearized rest points are D^-1(x) -- q =
 * D_pose^-1(x) in closed form, then p + u(p) = q by Newton's method, whose
 * root is unique because the field's Lipschitz bound (the root of the sum
 * over the axes of ((G-1) x the largest displacement difference along that
 * axis within a cell)^2, an upper bound of |du/dp|) is at most 0.9 -- and
 * the normal of a hit is J_D^-T n (Sec. 2.2); n_inst may not exceed the
 * field's instance count (NIF_ERR_ARG).
 * nif_set_field: n_inst fields of G nodes per axis, 2 <= G <= 33, from
 * delta_host [n_inst][G][G][G][3] (index [i][c][b][a], host, copied); the
 * Adam moments of the field are reset. NIF_ERR_ARG if a displacement is not
 * finite or a field's bound exceeds 0.9. n_inst == 0 removes the field.
 * A query plan applies the field as it was when the plan was created: while
 * plans exist, only the values of an existing field may change (same n_inst
 * and G), otherwise NIF_ERR_STATE. Synchronises the device.
 * nif_get_field: *n_inst_host and *G_host (nullable) receive the sizes;
 * delta_host (nullable, `bytes` = n_inst G^3 3 sizeof(float)) the values.
 * Synchronises the device. */
nif_status nif_set_field(nif_handle* h, int n_inst, int G, const float* delta_host);
nif_status nif_get_field(nif_handle* h, int* n_inst_host, int* G_host, float* delta_host, size_t bytes);

/* Gradient with respect to the field (FP32): for segments whose deformed end
 * points x0 = o + t0 d, x1 = o + t1 d are held fixed, the rest points are
 * p = D^-1(x); with q = D_pose^-1(x) fixed, p + u(p) = q gives
 * dp/d(delta_n) = -(I + du/dp)^-1 w_n(p), w_n the trilinear weight of node
 * n. With tables and weights frozen this adds d(sum dfeats * [psi(p0) (+)
 * psi(p1)])/d(delta) into dfield_dev [n_inst][G^3][3] (accumulated). Other
 * arguments as nif_pose_gradient. NIF_ERR_STATE without a field. */
nif_status nif_field_gradient(nif_handle* h, const nif_pose* poses_host, int n_inst,
                              const int* inst_offsets_dev, const nif_segment* segs_dev,
                              const nif_linseg* lin_dev, int64_t n, const float* dfeats_dev,
                              float* dfield_dev, void* stream);

/* One fitting step of the field against a target deformation (FP32 handles
 * of the composed encoding): the segments of rays_dev under the current
 * deformation (poses_host and the field; the batch rule of
 * nif_train_step_rays) are labelled along their rest segments under the
 * target deformation (target_poses_host, no field; Sec. 2's ground truth),
 * the task loss of Sec. 2.4 is taken on the network's outputs at the current
 * rest segments, and its gradient goes through the MLP, the encoding and
 * the field's inverse into the field: Adam (beta 0.9, 0.99; learning rate
 * lr_field) on the displacements, after which a field whose Lipschitz bound
 * passed 0.9 is scaled back onto it. With lr_grid or lr_mlp > 0 the network
 * is trained on the same loss in the same step (jointly); with both 0 it is
 * frozen. loss_host (nullable, blocks): the loss parts as nif_train_step
 * gives them. NIF_ERR_STATE without a field or on other handles. */
nif_status nif_field_step(nif_handle* h, const nif_pose* poses_host, int n_inst, const nif_ray* rays_dev,
                          const int* inst_offsets_dev, int n_rays, int64_t n_segments,
                          const nif_pose* target_poses_host, float lr_field, float lr_grid, float lr_mlp,
                          double* loss_host, void* stream);

/* Shadow rays for a frame loop (occlusion queries with NIF_SHADOW_ONLY):
 * for a primary ray that hit, origin o + D d, direction the normalised
 * light_dir_host, interval [eps, tmax]; for a miss an empty interval
 * [0, 0] (no segments, reported as no hit). shadow_rays_dev [n] may not
 * alias rays_dev. */
nif_status nif_shadow_rays(nif_handle* h, const nif_ray* rays_dev, const nif_hit* hits_dev, int n,
                           const float* light_dir_host, float eps, float tmax, nif_ray* shadow_rays_dev,
                           void* stream);

/* Draws the training rays of nif_train_step: rays_dev [n] for stream id
 * `stream_id` of step_seed (uniforms are the top 24 bits of splitmix64 of
 * (step_seed, stream_id, index)). */
nif_status nif_sample_rays(nif_handle* h, unsigned long long step_seed, int stream_id, int n,
                           nif_ray* rays_dev, void* stream);

/* Batched query as one CUDA graph. A plan binds the caller's device buffers
 * (n_rays rays split over n_inst instances by inst_offsets_dev, hits_dev)
 * and a segment capacity (seg_capacity <= 0: 1.5 x the segments of
 * poses_host), optionally autotunes the launch knobs on those buffers
 * (traversal warps per block, encoding block size and grid, rows per
 * encode + MLP chunk; the choice is kept in the handle and used by
 * nif_query too) and captures the whole query path -- pose upload, refit,
 * segments, linearization, encoding, MLP (cfg.precision), reconstruction --
 * with every element count kept on the device. nif_query_plan_create blocks;
 * nif_query_plan_run copies new poses into a pinned buffer (after the
 * previous replay of this plan finished) and launches the graph on
 * `stream` without further host synchronisation. Overflow of the segment
 * capacity is latched in the status word (nif_sync_status). The rays'
 * contents may change between runs; their buffers may not. A plan must be
 * destroyed before its handle. Other calls on the handle (queries, training,
 * further plans) may run between replays on the same stream: while a plan
 * lives, scratch that must grow is reallocated and the old allocation the
 * plan's graph uses is kept until the handle's last plan is destroyed. */
typedef struct nif_query_plan nif_query_plan;
nif_status nif_query_plan_create(nif_handle* h, int n_inst, const nif_ray* rays_dev,
                                 const int* inst_offsets_dev, int n_rays, nif_hit* hits_dev,
                                 int64_t seg_capacity, unsigned flags, int autotune,
                                 const nif_pose* poses_host, nif_query_plan** out);
nif_status nif_query_plan_run(nif_query_plan* plan, const nif_pose* poses_host, void* stream);
nif_status nif_query_plan_info(const nif_query_plan* plan, int* trav_warps, int* enc_threads,
                               int* enc_blocks_per_sm, int64_t* tc_chunk, int64_t* seg_capacity);
void nif_query_plan_destroy(nif_query_plan* plan);

/* Synchronises `stream` and returns (and clears) the device status word. */
nif_status nif_sync_status(nif_handle* h, void* stream);

/* Knobs of a handle, for failure testing and tuning (the paper has none).
 * NIF_KNOB_WAIT_NS: the bound, in nanoseconds, of the waits in the work
 *   loops of the tensor-core kernels (the MLP forward, backward and weight
 *   gradients): a wait that takes longer makes the kernel latch
 *   NIF_ERR_TIMEOUT in the status word, stop its work, wait (with the fixed
 *   one-second bound) for its own copies and tensor-core operations in
 *   flight, free its tensor memory and return; the outputs of that launch
 *   are then undefined and the handle stays usable. 0 restores the default,
 *   one second; the value must lie in [0, 6e10]. Synchronises the device.
 * NIF_KNOB_SEG_SCRATCH: scale in (0, 1] of the scratch into which one
 *   traversal writes the segments of a query or training batch before they
 *   are put in ray order (default 1); below 1 the scratch overflows sooner
 *   and the device-gated second traversal writes the rows instead. Results
 *   do not depend on it.
 * NIF_KNOB_QUERY_SEGS: segments per ray, in (0, 4096], that nif_query sizes
 *   its capacity for until a query's total has come back (default 8); setting
 *   it forgets the totals of earlier queries.
 * NIF_KNOB_BATCH_AT: where the next step's batch starts beside an FP32 step
 *   of nif_train_steps / nif_train_steps_rays: 0 with the step (default),
 *   1 after the encoding forward, 2 after the MLP forward, 3 after the MLP
 *   backward. A scheduling choice only: the steps compute the same.
 * NIF_KNOB_FP32_FUSED: 1 (default) runs every layer of the FP32 MLP forward
 *   in one persistent launch whose hidden activations stay in shared memory
 *   (a training step still writes the activations its backward reads; a
 *   query writes none), 0 one launch per layer, in training steps,
 *   nif_mlp_forward and queries alike. Applies to hidden widths 32 and 64
 *   with at least one hidden layer and in_dim a multiple of 4; the results
 *   are the same. An autotuned query plan of an FP32 handle times both and
 *   keeps the faster for its queries (the training steps keep the knob's).
 * NIF_KNOB_QUERY_FUSED: 1 (default) computes a BF16/FP16 query's encoding
 *   (Eq. 1) inside the tensor-core MLP's kernel, which keeps each tile's
 *   features in shared memory (handles with L in {4, 8, 16}, F_d = 2, width
 *   32 or 64 and an FP16 table copy of at most 4 MiB); 0 runs the encoding
 *   and the MLP as two kernels per chunk with the features in a global
 *   buffer. The outputs agree to the MLP's accumulation order and the fast
 *   sine of gamma. A query plan's autotuner times both and keeps the faster.
 * NIF_KNOB_STEP_PRIORITY: 1 runs the steps of nif_train_steps and
 *   nif_train_steps_rays on the handle's streams of the device's greatest
 *   priority (ordered after the caller's work and before its next), while
 *   the next batch is built on a stream of the least priority; 0 (default)
 *   runs them on the caller's stream. A scheduling choice only (measured on
 *   the 64^3 FP32 step: 3.06-3.09 ms with priorities, 3.04-3.05 ms without:
 *   a batch that finishes later delays the step that needs it).
 *   Synchronises the device.
 * NIF_KNOB_DEFER_WEIGHTS: 1 (default) lets an FP32 step of nif_train_steps
 *   / nif_train_steps_rays update the tables on the step's stream right
 *   after the encoding backward, and the MLP weights and log-variances on
 *   the handle's second stream after the weight gradients, beside the next
 *   step's encoding forward (which writes a second feature buffer); the next
 *   step's MLP forward waits for that update, and every call ends with all
 *   of it ordered on the caller's stream. 0 updates all parameters in one
 *   launch after both gradients. The same Adam arithmetic either way.
 *   Synchronises the device.
 * NIF_KNOB_STEP_FWD_CTAS: persistent CTAs of a training step's MLP forward
 *   (the one-launch FP32 forward or the 16-bit tensor-core forward) while
 *   nif_train_steps / nif_train_steps_rays build the next batch beside it.
 *   0 (default): the FP32 forward takes three quarters of the SMs, then the
 *   fewest CTAs that give each the same number of 128-row tiles, so that the
 *   batch's kernels keep the other SMs, and the 16-bit forward one CTA per
 *   SM; k > 0: k CTAs (at most one per SM); -1: one per SM. A scheduling
 *   choice only: the steps compute the same.
 * NIF_KNOB_STEP_BWD_CTAS: persistent CTAs of the encoding backward in an
 *   FP32 training step, which runs beside the weight gradients on the
 *   handle's second stream. 0 (default): seven eighths of the SMs, leaving
 *   the rest to the weight gradients; k > 0: k CTAs (at most one per SM);
 *   -1: one per SM (as in nif_encode_segments_backward and mixed-precision
 *   steps). A scheduling choice only: the same sums in another order.
 * NIF_KNOB_DETERMINISTIC: 1 makes the gradients of training steps (and of
 *   nif_encode_segments_backward) independent of the order in which the GPU
 *   adds them, so that the same calls on the same state give bit-identical
 *   parameters, losses and checkpoints, across runs and after a checkpoint
 *   is loaded into another handle; 0 (default) adds them with float
 *   reductions in L2, whose order varies from run to run. In this mode the
 *   table gradient is summed as 64-bit fixed point: each contribution is
 *   rounded once to a multiple of 2^-S, with S chosen per call from the
 *   largest dL/dfeature so that no sum can overflow, and each sum is
 *   converted to FP32 at the end (an added absolute error of at most 2^-(S+1)
 *   per contribution); the MLP weight gradients are summed per row range and
 *   the ranges added in order; the loss sums are added in block order. The
 *   paper has no counterpart (it trains with no stated reduction order).
 *   Slower (measured on the 64^3 FP32 step in the design notes). The
 *   gradients with respect to poses and to a learned field (nif_pose_step,
 *   nif_pose_gradient, nif_field_gradient and the field part of
 *   nif_field_step) keep their float reductions. Handles with
 *   NIF_FLAG_CONCAT_ENCODING are refused (NIF_ERR_ARG). Synchronises the
 *   device.
 * NIF_KNOB_ORDER_BITS: b in [4, 8] (default 7): the encoders of tables over
 *   4 MiB visit the distinct end points sorted by the Morton code of their
 *   cell in a 2^b-per-axis grid over the rest cube (a counting sort over
 *   2^(3b) cells), so that a warp's points share corner rows. A scheduling
 *   choice only: the features are the same. Synchronises the device.
 * NIF_KNOB_BWD_SPLIT: 1 or 2: how many tasks share a gamma term's levels in
 *   the run-length encoding backward (2: one task per half of the levels, so
 *   that a warp's 32 lanes hold the fine levels of 4 terms; for L with
 *   L/2 >= 4 dividing 32, else 1); 0 (default): 2 when L >= 16, else 1. A
 *   scheduling choice only: the same sums in another order.
 * NIF_KNOB_FAIL_ALLOC: n >= 1 makes the n-th allocation of scratch memory
 *   from now on (a buffer the handle grows on demand) fail as an
 *   out-of-memory cudaMalloc would: the call that needs it returns
 *   NIF_ERR_OOM and the buffer is left unallocated, to be allocated again
 *   by a later call. 0 (default) disables it. Host-side fault injection for
 *   testing recovery; nothing fails on the device. A training call that
 *   fails before its parameter update clears the gradients it had added,
 *   so the trainable state is the one before the call.
 * NIF_ERR_ARG for an unknown knob or a value out of range. */
#define NIF_KNOB_WAIT_NS 1
#define NIF_KNOB_SEG_SCRATCH 2
#define NIF_KNOB_QUERY_SEGS 3
#define NIF_KNOB_BATCH_AT 4
#define NIF_KNOB_FP32_FUSED 5
#define NIF_KNOB_QUERY_FUSED 6
#define NIF_KNOB_STEP_PRIORITY 7
#define NIF_KNOB_DEFER_WEIGHTS 8
#define NIF_KNOB_STEP_FWD_CTAS 9
#define NIF_KNOB_STEP_BWD_CTAS 10
#define NIF_KNOB_DETERMINISTIC 11
#define NIF_KNOB_ORDER_BITS 12
#define NIF_KNOB_FAIL_ALLOC 13
#define NIF_KNOB_BWD_SPLIT 14
nif_status nif_set_knob(nif_handle* h, int knob, double value);

/* Allocation-free variant of nif_segments (the paper has no counterpart:
 * this is an integration aid). For callers that cannot call cudaMalloc -- a
 * host application that owns all device memory through its own fixed-budget
 * allocator, or a latency-critical loop where cudaMalloc's implicit
 * device-wide synchronisation is not allowed. Same arguments, definition and
 * outputs as nif_segments; the caller passes every input and output buffer.
 * Its scratch (per-ray counts and scan block sums) lives in one file-scope
 * device array of (NIF_NOALLOC_MAX_RAYS + 2048) 32-bit words, about 4 MiB,
 * that every GPU loading the library holds until the process exits.
 * Limits: n_rays <= NIF_NOALLOC_MAX_RAYS and n_inst <= the number of
 * instances the handle already holds buffers for (1 after nif_create, more
 * after an allocating call with more instances); otherwise NIF_ERR_ARG.
 * The first call on a device looks the array's device address up (with that
 * device current). Every call shares the one array: calls that overlap on the
 * GPU (other streams, other handles, other threads) race and must be
 * serialised by the caller. Like nif_segments it blocks the host (it reads
 * the total back), so it must not be called while `stream` is being captured
 * into a CUDA graph. segs_dev == NULL only counts. */
#define NIF_NOALLOC_MAX_RAYS (1 << 20)
nif_status nif_segments_noalloc(nif_handle* h, const nif_pose* poses_host, int n_inst,
                                const nif_ray* rays_dev, const int* inst_offsets_dev, int n_rays,
                                uint32_t* ray_offsets_dev, nif_segment* segs_dev, int64_t seg_cap,
                                int64_t* n_segs_host, void* stream);

/* ------------------------------------------------------------------------ */
/* Diagnostics                                                               */
/* ------------------------------------------------------------------------ */

/* Number of kernels this library has enqueued since it was loaded (all
 * handles, all threads). */
unsigned long long nif_kernel_launches(void);

/* Bounds-checked build (the paper has none: a debugging aid). The library
 * compiled with -DNIF_BOUNDS=1 (libnif_bounds.so) checks the index
 * computations of its gathers and scatters -- the grid cell of every encoder
 * gather and scatter (so every table row stays inside its level), the
 * triangle indices of the labels, the positions of the rest-space point order
 * and of the per-ray segment rows -- and, when a check fails, counts it in a
 * device word and redirects or skips the access instead of trapping.
 * *enabled = 1 in that build (the call then synchronises the device and
 * returns in *failures the checks that failed since the last call, clearing
 * the count); *enabled = 0 and *failures = 0 in the normal build, whose checks
 * compile away. NIF_ERR_ARG for null pointers. */
nif_status nif_bounds_check(int* enabled, unsigned long long* failures);

/* Measured ceilings of the memory patterns that bound the encoding kernels
 * (the paper has no counterpart): `kind`
 *   NIF_PROBE_RED8   random red.global.add.v2.f32 (8-byte FP32 reductions,
 *                    the encoding backward's per-corner update),
 *   NIF_PROBE_RED16  random red.global.add.v4.f32 into two adjacent rows
 *                    (its paired x-edge corners),
 *   NIF_PROBE_LOAD8  random 8-byte row loads (FP32 table rows, the forward),
 *   NIF_PROBE_LOAD4  random 4-byte row loads (FP16 table rows),
 * each lane at its own random row (one 32-byte sector per access: the L2's
 * rate for scattered accesses), or, with the _WARP kinds, each warp's 32
 * lanes at 32 consecutive rows of a random block (whole sectors: the rate
 * when every fetched byte is used), over buf_dev (caller-owned, `bytes` = a power-of-two number >= 1024 of
 * rows, 16-byte aligned; its contents are changed by the reductions), which
 * stays in L2 when it fits: one warm-up launch, then 5 launches of
 * 8 x num_SMs blocks of 256 threads, each thread `iters` x 8 independent
 * accesses, timed with CUDA events on `stream`. *gbs_host receives the
 * payload bytes per second / 1e9, *ms_host the mean launch time. Blocks the
 * host. */
#define NIF_PROBE_RED8 1
#define NIF_PROBE_RED16 2
#define NIF_PROBE_LOAD8 3
#define NIF_PROBE_LOAD4 4
#define NIF_PROBE_RED8_WARP 5
#define NIF_PROBE_RED16_WARP 6
#define NIF_PROBE_LOAD8_WARP 7
#define NIF_PROBE_LOAD4_WARP 8
nif_status nif_probe_memory(nif_handle* h, int kind, void* buf_dev, size_t bytes, int iters, double* gbs_host,
                            double* ms_host, void* stream);
/* Distinct end points listed by the handle's last segment encoding (the
 * forward writes a repeated entry point's features from its previous exit
 * point's, and the backward walks the distinct points only) and the number
 * of segments it encoded. Blocks the host; NIF_ERR_STATE before any. */
nif_status nif_encoder_points(nif_handle* h, int64_t* n_points_host, int64_t* n_segments_host);

/* Per-stage timing: with profiling on, every stage the handle runs is
 * bracketed by two CUDA events on its stream (a few microseconds of
 * overhead per stage). nif_profile(h, 1) clears the record and turns it on,
 * nif_profile(h, 0) turns it off; both synchronise the device. */
nif_status nif_profile(nif_handle* h, int enable);
/* Restricts the per-stage timing to the stages named in `names`, a
 * comma-separated list of stage names as nif_profile_read reports them
 * (host string, copied); NULL or "" times every stage again. Fewer events
 * in a timed interval add less to it. Synchronises the device; NIF_ERR_ARG
 * for a list longer than 1024 characters. */
nif_status nif_profile_filter(nif_handle* h, const char* names);
/* Synchronises, folds the events into per-stage sums and returns entry i:
 * its name (copied into `name`, capacity name_cap), the summed milliseconds
 * and the number of timed launches of the stage; *n_names (nullable) gets
 * the number of stages. i = -1 only reports *n_names. */
nif_status nif_profile_read(nif_handle* h, int i, char* name, int name_cap, double* ms, long* count,
                            int* n_names);
/* The timed stages one by one, before nif_profile_read folds them: record i
 * (in launch order) gives its name and its start and end in milliseconds
 * after the start of record 0, on the GPU's clock (stages on different
 * streams overlap). *n_recs (nullable) gets the number of records; i = -1
 * only reports it. Synchronises the device; NIF_ERR_ARG for i out of range. */
nif_status nif_profile_timeline(nif_handle* h, int i, char* name, int name_cap, double* t0_ms, double* t1_ms,
                                int* n_recs);

#ifdef __cplusplus
}
#endif
#endif /* NIF_H */
