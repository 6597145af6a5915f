// nif_api.cu -- host side of the C ABI declared in include/nif.h: handle
// lifetime, parameter I/O, the octree topology, and the orchestration of the
// query and training paths over the kernels of the k_*.cu files.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "nif_internal.cuh"

#include <atomic>

static thread_local std::string g_create_err;
static std::atomic<unsigned long long> g_launches{0};

void nif_count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }

extern "C" unsigned long long nif_kernel_launches(void) { return g_launches.load(); }

static bool prof_selected(const std::string& filter, const char* name) {
    if (filter.empty()) return true;
    const size_t n = std::strlen(name);
    size_t at = 0;
    while (at <= filter.size()) {
        size_t end = filter.find(',', at);
        if (end == std::string::npos) end = filter.size();
        if (end - at == n && filter.compare(at, n, name) == 0) return true;
        at = end + 1;
    }
    return false;
}

// Every stage is also an NVTX range on the calling host thread (header-only
// NVTX 3: a no-op unless a tool such as ncu --nvtx is attached), so a
// profiler can select one stage's launches by name.
NifProf::NifProf(nif_handle* h_, const char* name, cudaStream_t s_) : h(h_), s(s_) {
    nvtxRangePushA(name);
    if (!h || !h->prof || !prof_selected(h->prof_filter, name)) return;
    if (h->prof_used + 2 > h->prof_pool.size()) {
        for (int i = 0; i < 64; i++) {
            cudaEvent_t e;
            if (cudaEventCreate(&e) != cudaSuccess) return;
            h->prof_pool.push_back(e);
        }
    }
    nif_handle::ProfRec r{name, h->prof_pool[h->prof_used], h->prof_pool[h->prof_used + 1]};
    h->prof_used += 2;
    cudaEventRecord(r.a, s);
    rec = h->prof_recs.size();
    h->prof_recs.push_back(r);
}

NifProf::~NifProf() {
    if (rec != (size_t)-1) cudaEventRecord(h->prof_recs[rec].b, s);
    nvtxRangePop();
}

extern "C" nif_status nif_profile(nif_handle* h, int enable) {
    if (!h) return NIF_ERR_ARG;
    NIF_CK(h, cudaDeviceSynchronize());
    h->prof = enable != 0;
    h->prof_recs.clear();
    h->prof_used = 0;
    h->prof_sum.clear();
    return NIF_OK;
}

extern "C" nif_status nif_profile_filter(nif_handle* h, const char* names) {
    if (!h) return NIF_ERR_ARG;
    if (names && std::strlen(names) > 1024) return nif_fail(h, NIF_ERR_ARG, "profile filter longer than 1024");
    NIF_CK(h, cudaDeviceSynchronize());
    h->prof_filter = names ? names : "";
    return NIF_OK;
}

// fold the recorded events into per-name sums (synchronises)
static nif_status prof_fold(nif_handle* h) {
    NIF_CK(h, cudaDeviceSynchronize());
    for (auto& r : h->prof_recs) {
        float ms = 0.f;
        NIF_CK(h, cudaEventElapsedTime(&ms, r.a, r.b));
        bool found = false;
        for (auto& p : h->prof_sum)
            if (p.first == r.name) { p.second.first += ms; p.second.second += 1; found = true; break; }
        if (!found) h->prof_sum.push_back({r.name, {(double)ms, 1L}});
    }
    h->prof_recs.clear();
    h->prof_used = 0;
    return NIF_OK;
}

extern "C" nif_status nif_profile_timeline(nif_handle* h, int i, char* name, int name_cap, double* t0_ms,
                                           double* t1_ms, int* n_recs) {
    if (!h) return NIF_ERR_ARG;
    NIF_CK(h, cudaDeviceSynchronize());
    if (n_recs) *n_recs = (int)h->prof_recs.size();
    if (i == -1) return NIF_OK;
    if (i < 0 || i >= (int)h->prof_recs.size()) return NIF_ERR_ARG;
    const nif_handle::ProfRec& r0 = h->prof_recs[0];
    const nif_handle::ProfRec& r = h->prof_recs[i];
    float a = 0.f, b = 0.f;
    NIF_CK(h, cudaEventElapsedTime(&a, r0.a, r.a));
    NIF_CK(h, cudaEventElapsedTime(&b, r0.a, r.b));
    if (name && name_cap > 0) {
        std::strncpy(name, r.name, name_cap - 1);
        name[name_cap - 1] = 0;
    }
    if (t0_ms) *t0_ms = a;
    if (t1_ms) *t1_ms = b;
    return NIF_OK;
}

extern "C" nif_status nif_profile_read(nif_handle* h, int i, char* name, int name_cap, double* ms, long* count,
                                       int* n_names) {
    if (!h) return NIF_ERR_ARG;
    nif_status st = prof_fold(h);
    if (st != NIF_OK) return st;
    if (n_names) *n_names = (int)h->prof_sum.size();
    if (i < 0 || i >= (int)h->prof_sum.size()) return i == -1 ? NIF_OK : NIF_ERR_ARG;
    if (name && name_cap > 0) {
        std::strncpy(name, h->prof_sum[i].first.c_str(), name_cap - 1);
        name[name_cap - 1] = 0;
    }
    if (ms) *ms = h->prof_sum[i].second.first;
    if (count) *count = h->prof_sum[i].second.second;
    return NIF_OK;
}

nif_status nif_fail(nif_handle* h, nif_status st, const std::string& msg) {
    if (h) h->err = msg;
    else g_create_err = msg;
    return st;
}

nif_status nif_cuda_fail(nif_handle* h, cudaError_t e, const char* what) {
    std::string m = std::string(what) + ": " + cudaGetErrorString(e);
    return nif_fail(h, e == cudaErrorMemoryAllocation ? NIF_ERR_OOM : NIF_ERR_CUDA, m);
}

void nif_retire(nif_handle* h, void* p) {
    if (!p) return;
    if (h->n_plans > 0) h->graveyard.push_back(p);
    else cudaFree(p);
}

void nif_free_retired(nif_handle* h) {
    if (h->graveyard.empty()) return;
    cudaDeviceSynchronize();
    for (void* p : h->graveyard) cudaFree(p);
    h->graveyard.clear();
}

nif_status nif_grow(nif_handle* h, nif_handle::Buf& b, size_t bytes) {
    if (bytes <= b.bytes) return NIF_OK;
    if (b.p) {
        NIF_CK(h, cudaDeviceSynchronize());
        nif_retire(h, b.p);
        b.p = nullptr;
        b.bytes = 0;
    }
    size_t want = bytes + bytes / 4 + 256;
    if (h->fail_alloc > 0 && --h->fail_alloc == 0)
        return nif_fail(h, NIF_ERR_OOM, "cudaMalloc(scratch): injected failure (NIF_KNOB_FAIL_ALLOC)");
    cudaError_t e = cudaMalloc(&b.p, want);
    if (e != cudaSuccess) {
        cudaGetLastError();
        b.p = nullptr;
        return nif_cuda_fail(h, e, "cudaMalloc(scratch)");
    }
    b.bytes = want;
    return NIF_OK;
}

// ---------------------------------------------------------------------------
// Small kernels of the host orchestration
// ---------------------------------------------------------------------------
namespace {

__global__ void k_to_lowp(const float* __restrict__ src, size_t n, __half* __restrict__ h16,
                          __nv_bfloat16* __restrict__ b16) {
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        float v = src[i];
        if (h16) h16[i] = __float2half_rn(v);
        if (b16) b16[i] = __float2bfloat16_rn(v);
    }
}

// transposed 16-bit copies of the weight matrices: layer l [out_l][in_l] -> [in_l][out_l]
struct LayerDims {
    int n;
    size_t off[NIF_MAX_LAYERS + 1];   // element offsets relative to layer 0
    int in[NIF_MAX_LAYERS], out[NIF_MAX_LAYERS];
};

__global__ void k_to_lowp_t(const float* __restrict__ w, LayerDims d, __half* __restrict__ h16,
                            __nv_bfloat16* __restrict__ b16) {
    const size_t total = d.off[d.n];
    for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
        int l = 0;
        while (l + 1 < d.n && e >= d.off[l + 1]) l++;
        const size_t r = e - d.off[l];
        if (r >= (size_t)d.in[l] * d.out[l]) continue;      // alignment padding between layers
        const int o = (int)(r / d.in[l]), i = (int)(r % d.in[l]);
        const float v = w[e];
        const size_t t = d.off[l] + (size_t)i * d.out[l] + o;
        h16[t] = __float2half_rn(v);
        b16[t] = __float2bfloat16_rn(v);
    }
}

// up to kPoseArg poses passed by value (the kernel-argument block holds 4 KB)
constexpr int kPoseArg = 128;
struct PoseArg {
    int n;
    float4 p[kPoseArg];
};

__global__ void k_set_poses(PoseArg a, float4* __restrict__ d) {
    if ((int)threadIdx.x < a.n) d[threadIdx.x] = a.p[threadIdx.x];
}

// offsets[i] = i * per for i <= n
__global__ void k_iota_offsets(int* __restrict__ offsets, int n, int per) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i <= n) offsets[i] = i * per;
}

uint64_t mix64(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// splitmix64 stream output `counter` of `seed` as a uniform in [0,1) (24 bits)
float host_uniform(uint64_t seed, uint64_t counter) {
    uint64_t z = mix64(seed + (counter + 1ull) * 0x9E3779B97F4A7C15ull);
    return (float)(z >> 40) * (1.0f / 16777216.0f);
}

uint32_t morton3(uint32_t i, uint32_t j, uint32_t k) {
    auto spread = [](uint32_t x) {
        x &= 0x3ff;
        x = (x | (x << 16)) & 0x030000FF;
        x = (x | (x << 8)) & 0x0300F00F;
        x = (x | (x << 4)) & 0x030C30C3;
        x = (x | (x << 2)) & 0x09249249;
        return x;
    };
    return spread(i) | (spread(j) << 1) | (spread(k) << 2);
}

}  // namespace

nif_status nif_refresh_lowp(nif_handle* h, cudaStream_t s) {
    if (!h->lowp_dirty) return NIF_OK;
    size_t nt = (size_t)h->L * h->T * h->Fd;
    k_to_lowp<<<std::max(1, std::min(h->num_sms * 8, (int)((nt + 255) / 256))), 256, 0, s>>>(
        h->d_params + h->off_tables, nt, h->d_tables_h, nullptr);
    NIF_CK_LAUNCH(h);
    size_t nw = h->off_s - h->off_layer[0];
    k_to_lowp<<<std::max(1, std::min(h->num_sms * 8, (int)((nw + 255) / 256))), 256, 0, s>>>(
        h->d_params + h->off_layer[0], nw, h->d_w_f16, h->d_w_bf16);
    NIF_CK_LAUNCH(h);
    LayerDims d{};
    d.n = h->n_layers;
    for (int l = 0; l <= h->n_layers; l++) d.off[l] = h->off_layer[l] - h->off_layer[0];
    for (int l = 0; l < h->n_layers; l++) {
        d.in[l] = h->lay_in[l];
        d.out[l] = h->lay_out[l];
    }
    k_to_lowp_t<<<std::max(1, std::min(h->num_sms * 4, (int)((nw + 255) / 256))), 256, 0, s>>>(
        h->d_params + h->off_layer[0], d, h->d_wt_f16, h->d_wt_bf16);
    NIF_CK_LAUNCH(h);
    h->lowp_dirty = false;
    return NIF_OK;
}

nif_status reset_loss_scale(nif_handle* h) {
    NifLossScale ls{h->cfg.precision == NIF_FP16 ? 32768.0f : 1.0f, 0, 0, 0, 1.0, 1.0,
                    (float)(1.0 / (1.0 - 0.9)), (float)(1.0 / (1.0 - 0.99))};
    NIF_CK(h, cudaMemcpy(h->d_ls, &ls, sizeof(ls), cudaMemcpyHostToDevice));
    return NIF_OK;
}

nif_status nif_ensure_instances(nif_handle* h, int n_inst) {
    if (n_inst <= h->inst_cap) return NIF_OK;
    NIF_CK(h, cudaDeviceSynchronize());
    nif_retire(h, h->d_corners);
    nif_retire(h, h->d_aabb);
    nif_retire(h, h->d_pose);
    h->d_corners = nullptr;
    h->d_aabb = nullptr;
    h->d_pose = nullptr;
    int cap = std::max(n_inst, 1);
    NIF_CK(h, cudaMalloc(&h->d_corners, sizeof(float) * 24 * (size_t)std::max(h->n_leaves, 1) * cap));
    NIF_CK(h, cudaMalloc(&h->d_aabb, sizeof(float4) * 2 * (size_t)std::max(h->n_nodes, 1) * cap));
    NIF_CK(h, cudaMalloc(&h->d_pose, sizeof(float4) * cap));
    h->inst_cap = cap;
    return NIF_OK;
}

nif_status nif_upload_poses(nif_handle* h, const nif_pose* poses, int n_inst, cudaStream_t s) {
    nif_status st = nif_ensure_instances(h, n_inst);
    if (st != NIF_OK) return st;
    if (n_inst <= kPoseArg) {
        // small batches travel as a kernel argument: no host round trip
        PoseArg a;
        a.n = n_inst;
        for (int i = 0; i < n_inst; i++)
            a.p[i] = make_float4(NIF_KBEND * poses[i].bend, poses[i].twist, poses[i].taper, 0.f);
        k_set_poses<<<1, kPoseArg, 0, s>>>(a, h->d_pose);
        NIF_CK_LAUNCH(h);
        return NIF_OK;
    }
    // larger batches go through a pinned staging buffer; it is rewritten only
    // once the previous copy from it has completed (an event, not a stream sync)
    if (h->pose_pending) NIF_CK(h, cudaEventSynchronize(h->ev_pose));
    h->pose_pending = false;
    if (n_inst > h->pose_pinned_cap) {
        if (h->h_pose_pinned) cudaFreeHost(h->h_pose_pinned);
        h->h_pose_pinned = nullptr;
        h->pose_pinned_cap = 0;
        NIF_CK(h, cudaMallocHost(&h->h_pose_pinned, sizeof(float4) * (size_t)n_inst));
        h->pose_pinned_cap = n_inst;
    }
    for (int i = 0; i < n_inst; i++)
        h->h_pose_pinned[i] = make_float4(NIF_KBEND * poses[i].bend, poses[i].twist, poses[i].taper, 0.f);
    NIF_CK(h, cudaMemcpyAsync(h->d_pose, h->h_pose_pinned, sizeof(float4) * n_inst, cudaMemcpyHostToDevice, s));
    NIF_CK(h, cudaEventRecord(h->ev_pose, s));
    h->pose_pending = true;
    return NIF_OK;
}

// ---------------------------------------------------------------------------
// Lifetime
// ---------------------------------------------------------------------------
static nif_status validate(const nif_config* c, const nif_mesh* m) {
    if (!c || !m) return nif_fail(nullptr, NIF_ERR_ARG, "null config or mesh");
    if (c->voxel_res < 2 || c->voxel_res > 512 || (c->voxel_res & (c->voxel_res - 1)))
        return nif_fail(nullptr, NIF_ERR_ARG, "voxel_res must be a power of two in [2, 512]");
    if (c->pe_bands < 0 || c->pe_bands > 8) return nif_fail(nullptr, NIF_ERR_ARG, "pe_bands in [0, 8]");
    if (c->levels < 1 || c->levels > NIF_MAX_LEVELS) return nif_fail(nullptr, NIF_ERR_ARG, "levels in [1, 32]");
    if (c->feats != 2) return nif_fail(nullptr, NIF_ERR_ARG, "feats must be 2");
    if (c->log2_table < 4 || c->log2_table > 24) return nif_fail(nullptr, NIF_ERR_ARG, "log2_table in [4, 24]");
    if (c->base_res < 1 || !(c->growth >= 1.0f)) return nif_fail(nullptr, NIF_ERR_ARG, "base_res >= 1, growth >= 1");
    if (c->mlp_depth < 1 || c->mlp_depth > NIF_MAX_LAYERS - 2) return nif_fail(nullptr, NIF_ERR_ARG, "mlp_depth in [1, 8]");
    if (c->mlp_width != 16 && c->mlp_width != 32 && c->mlp_width != 64 && c->mlp_width != 128)
        return nif_fail(nullptr, NIF_ERR_ARG, "mlp_width in {16, 32, 64, 128}");
    if (c->n_materials < 1 || c->n_materials > 8) return nif_fail(nullptr, NIF_ERR_ARG, "n_materials in [1, 8]");
    if (c->precision < NIF_FP32 || c->precision > NIF_FP16) return nif_fail(nullptr, NIF_ERR_ARG, "precision");
    if (c->flags & ~(NIF_FLAG_FIXED_TASK_WEIGHTS | NIF_FLAG_SIGMOID_DISTANCE | NIF_FLAG_MIXED_TRAINING |
                     NIF_FLAG_CONCAT_ENCODING | NIF_FLAG_BILINEAR_FACES))
        return nif_fail(nullptr, NIF_ERR_ARG, "unknown flags");
    if ((c->flags & NIF_FLAG_MIXED_TRAINING) && c->precision == NIF_FP32)
        return nif_fail(nullptr, NIF_ERR_ARG, "NIF_FLAG_MIXED_TRAINING needs precision NIF_BF16 or NIF_FP16");
    if (m->n_tris < 0 || m->n_verts < 0 || (m->n_tris > 0 && (!m->tris || !m->verts)))
        return nif_fail(nullptr, NIF_ERR_ARG, "mesh arrays");
    for (int t = 0; t < m->n_tris * 3; t++)
        if (m->tris[t] < 0 || m->tris[t] >= m->n_verts) return nif_fail(nullptr, NIF_ERR_ARG, "triangle index out of range");
    if (m->tri_material)
        for (int t = 0; t < m->n_tris; t++)
            if (m->tri_material[t] >= c->n_materials) return nif_fail(nullptr, NIF_ERR_ARG, "material out of range");
    for (int v = 0; v < m->n_verts * 3; v++)
        if (!(m->verts[v] >= 0.0f && m->verts[v] <= 1.0f)) return nif_fail(nullptr, NIF_ERR_ARG, "vertices must lie in [0,1]^3");
    return NIF_OK;
}

static nif_status build_octree(nif_handle* h) {
    int N = h->N;
    int64_t nvox = (int64_t)N * N * N;
    std::vector<uint8_t> occ(nvox);
    NIF_CK(h, cudaMemcpy(occ.data(), h->d_occ, nvox, cudaMemcpyDeviceToHost));
    std::vector<std::pair<uint32_t, uint32_t>> leaves;   // (morton, voxel)
    for (int64_t v = 0; v < nvox; v++)
        if (occ[v]) {
            uint32_t i = v % N, j = (v / N) % N, k = (uint32_t)(v / ((int64_t)N * N));
            leaves.push_back({morton3(i, j, k), (uint32_t)v});
        }
    std::sort(leaves.begin(), leaves.end());
    int n = (int)leaves.size();
    h->n_leaves = n;
    std::vector<uint32_t> vox(n), lat(n);
    for (int q = 0; q < n; q++) {
        uint32_t v = leaves[q].second;
        uint32_t i = v % N, j = (v / N) % N, k = v / (N * N);
        vox[q] = v;
        lat[q] = i | (j << 10) | (k << 20);
    }
    // internal levels: group nodes sharing the Morton prefix one octree level up
    std::vector<uint32_t> codes(n);
    for (int q = 0; q < n; q++) codes[q] = leaves[q].first;
    std::vector<int2> child;
    int level_first = 0;      // global index of the current level's first node
    int level_n = n;
    int next_global = n;
    h->level_begin.clear();
    h->level_count.clear();
    while (level_n > 8) {
        std::vector<uint32_t> pcodes;
        int begin = next_global;
        for (int q = 0; q < level_n;) {
            uint32_t pc = codes[q] >> 3;
            int r = q;
            while (r < level_n && (codes[r] >> 3) == pc) r++;
            child.push_back(make_int2(level_first + q, r - q));
            pcodes.push_back(pc);
            q = r;
        }
        int cnt = (int)pcodes.size();
        h->level_begin.push_back(begin);
        h->level_count.push_back(cnt);
        codes.swap(pcodes);
        level_first = begin;
        level_n = cnt;
        next_global = begin + cnt;
    }
    h->n_nodes = next_global;
    h->top_begin = level_first;
    h->top_count = level_n;
    NIF_CK(h, cudaMalloc(&h->d_leaf_vox, sizeof(uint32_t) * std::max(n, 1)));
    NIF_CK(h, cudaMalloc(&h->d_leaf_lat, sizeof(uint32_t) * std::max(n, 1)));
    NIF_CK(h, cudaMalloc(&h->d_child, sizeof(int2) * std::max((size_t)1, child.size())));
    if (n) {
        NIF_CK(h, cudaMemcpy(h->d_leaf_vox, vox.data(), sizeof(uint32_t) * n, cudaMemcpyHostToDevice));
        NIF_CK(h, cudaMemcpy(h->d_leaf_lat, lat.data(), sizeof(uint32_t) * n, cudaMemcpyHostToDevice));
    }
    if (!child.empty())
        NIF_CK(h, cudaMemcpy(h->d_child, child.data(), sizeof(int2) * child.size(), cudaMemcpyHostToDevice));
    return NIF_OK;
}

static nif_status init_params(nif_handle* h) {
    std::vector<float> p(h->n_params, 0.f);
    uint64_t seed = h->cfg.seed;
    uint64_t ctr = 0;
    size_t nt = (size_t)h->L * h->T * h->Fd;
    for (size_t i = 0; i < nt; i++) p[h->off_tables + i] = (2.0f * host_uniform(seed, ctr++) - 1.0f) * 1e-4f;
    for (int l = 0; l < h->n_layers; l++) {
        float b = std::sqrt(6.0f / (float)h->lay_in[l]);
        for (int o = 0; o < h->lay_out[l]; o++)
            for (int i = 0; i < h->lay_in[l]; i++) {
                float v = (2.0f * host_uniform(seed, ctr++) - 1.0f) * b;
                bool pad = (l == h->n_layers - 1) && o >= 8 + h->cfg.n_materials;
                p[h->off_layer[l] + (size_t)o * h->lay_in[l] + i] = pad ? 0.f : v;
            }
    }
    NIF_CK(h, cudaMemcpy(h->d_params, p.data(), sizeof(float) * h->n_params, cudaMemcpyHostToDevice));
    h->lowp_dirty = true;
    h->x3_dirty = true;
    return NIF_OK;
}

extern "C" nif_status nif_create(const nif_config* cfg, const nif_mesh* mesh, nif_handle** out) {
    if (!out) return nif_fail(nullptr, NIF_ERR_ARG, "null out");
    *out = nullptr;
    nif_status st = validate(cfg, mesh);
    if (st != NIF_OK) return st;
    nif_handle* h = new nif_handle();
    h->cfg = *cfg;
    h->N = cfg->voxel_res;
    h->L = cfg->levels;
    h->Fd = cfg->feats;
    h->P = 1 + 2 * cfg->pe_bands;
    h->T = 1u << cfg->log2_table;
    h->W = cfg->mlp_width;
    h->H = cfg->mlp_depth;
    h->n_layers = h->H + 1;
    h->concat = (cfg->flags & NIF_FLAG_CONCAT_ENCODING) != 0;
    h->point_w = h->concat ? 3 * h->P + h->L * h->Fd : h->P * h->L * h->Fd;
    h->in_dim = h->concat ? (2 * h->point_w + 15) / 16 * 16 : 2 * h->point_w;
    h->grid.L = h->L;
    h->grid.Fd = h->Fd;
    h->grid.P = h->P;
    h->grid.F = cfg->pe_bands;
    h->grid.T = h->T;
    h->grid.dense_mask = 0;
    for (int l = 0; l < h->L; l++) {
        double r = std::floor((double)cfg->base_res * std::pow((double)cfg->growth, (double)l));
        if (r > 1.0e6) { delete h; return nif_fail(nullptr, NIF_ERR_ARG, "level resolution too large"); }
        h->grid.res[l] = (int)r;
        double v = (r + 1.0) * (r + 1.0) * (r + 1.0);
        if (v <= (double)h->T) h->grid.dense_mask |= 1u << l;
    }
    int dev = 0;
    auto fail = [&](nif_status s) {
        g_create_err = h->err;
        nif_destroy(h);
        return s;
    };
    if (cudaGetDevice(&dev) != cudaSuccess) { delete h; return nif_fail(nullptr, NIF_ERR_CUDA, "no CUDA device"); }
    cudaDeviceGetAttribute(&h->num_sms, cudaDevAttrMultiProcessorCount, dev);
    if (h->num_sms <= 0) h->num_sms = 1;

    // mesh
    h->n_verts = mesh->n_verts;
    h->n_tris = mesh->n_tris;
    {
        std::vector<float> alb(3 * (size_t)std::max(h->n_tris, 1), 0.5f);
        std::vector<uint8_t> mat((size_t)std::max(h->n_tris, 1), 0);
        if (mesh->tri_albedo) std::memcpy(alb.data(), mesh->tri_albedo, sizeof(float) * 3 * h->n_tris);
        if (mesh->tri_material) std::memcpy(mat.data(), mesh->tri_material, h->n_tris);
#define CKC(call) do { cudaError_t e_ = (call); if (e_ != cudaSuccess) return fail(nif_cuda_fail(h, e_, #call)); } while (0)
        CKC(cudaMalloc(&h->d_verts, sizeof(float) * 3 * std::max(h->n_verts, 1)));
        CKC(cudaMalloc(&h->d_tris, sizeof(int) * 3 * std::max(h->n_tris, 1)));
        CKC(cudaMalloc(&h->d_alb, sizeof(float) * alb.size()));
        CKC(cudaMalloc(&h->d_mat, mat.size()));
        if (h->n_verts) CKC(cudaMemcpy(h->d_verts, mesh->verts, sizeof(float) * 3 * h->n_verts, cudaMemcpyHostToDevice));
        if (h->n_tris) CKC(cudaMemcpy(h->d_tris, mesh->tris, sizeof(int) * 3 * h->n_tris, cudaMemcpyHostToDevice));
        CKC(cudaMemcpy(h->d_alb, alb.data(), sizeof(float) * alb.size(), cudaMemcpyHostToDevice));
        CKC(cudaMemcpy(h->d_mat, mat.data(), mat.size(), cudaMemcpyHostToDevice));
        CKC(cudaMalloc(&h->d_tri_geo, sizeof(float4) * 3 * (size_t)std::max(h->n_tris, 1)));
        if (nif_tri_geo_run(h, nullptr) != NIF_OK) return fail(NIF_ERR_CUDA);
        CKC(cudaDeviceSynchronize());
    }
    CKC(cudaMalloc(&h->d_status, sizeof(int) * 4));
    CKC(cudaMemset(h->d_status, 0, sizeof(int) * 4));
    CKC(cudaMalloc(&h->d_lossacc, sizeof(double) * 16));
    CKC(cudaMemset(h->d_lossacc, 0, sizeof(double) * 16));
    CKC(cudaMalloc(&h->d_count, sizeof(int) * 4));
    CKC(cudaMemset(h->d_count, 0, sizeof(int) * 4));
    CKC(cudaMalloc(&h->d_next, sizeof(uint32_t) * 4));
    CKC(cudaMallocHost(&h->h_pinned, sizeof(int) * 16));
    CKC(cudaStreamCreateWithFlags(&h->aux, cudaStreamNonBlocking));
    {
        int least = 0, greatest = 0;
        CKC(cudaDeviceGetStreamPriorityRange(&least, &greatest));
        CKC(cudaStreamCreateWithPriority(&h->aux2, cudaStreamNonBlocking, least));
        CKC(cudaStreamCreateWithPriority(&h->hi, cudaStreamNonBlocking, greatest));
        CKC(cudaStreamCreateWithPriority(&h->aux_hi, cudaStreamNonBlocking, greatest));
    }
    CKC(cudaEventCreateWithFlags(&h->ev_hi_fork, cudaEventDisableTiming));
    CKC(cudaEventCreateWithFlags(&h->ev_wupd, cudaEventDisableTiming));
    CKC(cudaEventCreateWithFlags(&h->ev_dw[0], cudaEventDisableTiming));
    CKC(cudaEventCreateWithFlags(&h->ev_dw[1], cudaEventDisableTiming));
    CKC(cudaEventCreateWithFlags(&h->ev_hi_join, cudaEventDisableTiming));
    CKC(cudaEventCreateWithFlags(&h->ev_batch, cudaEventDisableTiming));
    CKC(cudaEventCreateWithFlags(&h->ev_step, cudaEventDisableTiming));
    CKC(cudaEventCreateWithFlags(&h->ev_fork, cudaEventDisableTiming));
    CKC(cudaEventCreateWithFlags(&h->ev_join, cudaEventDisableTiming));
    CKC(cudaEventCreateWithFlags(&h->ev_qtotal, cudaEventDisableTiming));
    CKC(cudaEventCreateWithFlags(&h->ev_pose, cudaEventDisableTiming));
    CKC(cudaMallocHost(&h->h_qtotal, sizeof(uint32_t) * 2));

    st = nif_voxelize_run(h);
    if (st != NIF_OK) return fail(st);
    st = build_octree(h);
    if (st != NIF_OK) return fail(st);

    // parameter layout
    size_t off = 0;
    h->off_tables = 0;
    off += (size_t)h->L * h->T * h->Fd;
    for (int l = 0; l < h->n_layers; l++) {
        h->lay_in[l] = l == 0 ? h->in_dim : h->W;
        h->lay_out[l] = l == h->n_layers - 1 ? NIF_OUT : h->W;
        off = (off + 7) & ~(size_t)7;     // 16-byte aligned rows in the 16-bit copies
        h->off_layer[l] = off;
        off += (size_t)h->lay_in[l] * h->lay_out[l];
    }
    off = (off + 7) & ~(size_t)7;
    h->off_layer[h->n_layers] = off;
    h->off_s = off;
    off += 8;
    h->n_params = off;
    CKC(cudaMalloc(&h->d_params, sizeof(float) * off));
    CKC(cudaMalloc(&h->d_grad, sizeof(float) * off));
    CKC(cudaMalloc(&h->d_m, sizeof(float) * off));
    CKC(cudaMalloc(&h->d_v, sizeof(float) * off));
    CKC(cudaMemset(h->d_grad, 0, sizeof(float) * off));
    CKC(cudaMemset(h->d_m, 0, sizeof(float) * off));
    CKC(cudaMemset(h->d_v, 0, sizeof(float) * off));
    CKC(cudaMalloc(&h->d_tables_h, sizeof(__half) * (size_t)h->L * h->T * h->Fd));
    CKC(cudaMalloc(&h->d_w_bf16, sizeof(__nv_bfloat16) * (h->off_s - h->off_layer[0])));
    CKC(cudaMalloc(&h->d_w_f16, sizeof(__half) * (h->off_s - h->off_layer[0])));
    CKC(cudaMalloc(&h->d_wt_bf16, sizeof(__nv_bfloat16) * (h->off_s - h->off_layer[0])));
    CKC(cudaMalloc(&h->d_wt_f16, sizeof(__half) * (h->off_s - h->off_layer[0])));
    CKC(cudaMemset(h->d_wt_bf16, 0, sizeof(__nv_bfloat16) * (h->off_s - h->off_layer[0])));
    CKC(cudaMemset(h->d_wt_f16, 0, sizeof(__half) * (h->off_s - h->off_layer[0])));
    CKC(cudaMalloc(&h->d_ls, sizeof(NifLossScale)));
#undef CKC
    if ((st = nif_x3_alloc(h)) != NIF_OK) return fail(st);
    if ((st = reset_loss_scale(h)) != NIF_OK) return fail(st);
    st = init_params(h);
    if (st != NIF_OK) return fail(st);
    st = nif_ensure_instances(h, 1);
    if (st != NIF_OK) return fail(st);
    *out = h;
    return NIF_OK;
}

extern "C" void nif_destroy(nif_handle* h) {
    if (!h) return;
    cudaDeviceSynchronize();
    void* ptrs[] = {h->d_verts, h->d_tris, h->d_tri_geo, h->d_alb, h->d_mat, h->d_occ, h->d_tri_ptr, h->d_tri_idx, h->d_child,
                    h->d_leaf_vox, h->d_leaf_lat, h->d_corners, h->d_aabb, h->d_pose, h->d_params, h->d_grad,
                    h->d_m, h->d_v, h->d_tables_h, h->d_w_bf16, h->d_w_f16, h->d_wt_bf16, h->d_wt_f16, h->d_ls,
                    h->d_w_x3, h->d_vox_leaf, h->d_status, h->d_lossacc, h->d_count,
                    h->d_next};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    nif_handle::Buf* bufs[] = {&h->b_counts, &h->b_offsets, &h->b_segs, &h->b_lin, &h->b_feat, &h->b_out,
                               &h->b_acts, &h->b_dout, &h->b_dx, &h->b_labels, &h->b_scan, &h->b_rays,
                               &h->b_inst, &h->b_feat2, &h->b_temp, &h->b_dys, &h->b_dup, &h->b_pts,
                               &h->b_lattice, &h->b_sort, &h->b_lin_t, &h->b_feat_alt, &h->b_fix, &h->b_parts, &h->b_lparts, &h->alt_counts, &h->alt_offsets, &h->alt_temp, &h->alt_segs,
                               &h->alt_scan, &h->alt_rays, &h->alt_inst, &h->alt_lin, &h->alt_labels,
                               &h->alt_dup, &h->alt_pts, &h->alt_sort};
    for (auto* b : bufs)
        if (b->p) cudaFree(b->p);
    if (h->h_pinned) cudaFreeHost(h->h_pinned);
    if (h->h_qtotal) cudaFreeHost(h->h_qtotal);
    if (h->h_pose_pinned) cudaFreeHost(h->h_pose_pinned);
    if (h->d_chunk_counts) cudaFree(h->d_chunk_counts);
    if (h->ev_qtotal) cudaEventDestroy(h->ev_qtotal);
    if (h->ev_pose) cudaEventDestroy(h->ev_pose);
    if (h->ev_fork) cudaEventDestroy(h->ev_fork);
    if (h->ev_join) cudaEventDestroy(h->ev_join);
    if (h->aux) cudaStreamDestroy(h->aux);
    if (h->aux2) cudaStreamDestroy(h->aux2);
    if (h->hi) cudaStreamDestroy(h->hi);
    if (h->aux_hi) cudaStreamDestroy(h->aux_hi);
    if (h->ev_hi_fork) cudaEventDestroy(h->ev_hi_fork);
    if (h->ev_wupd) cudaEventDestroy(h->ev_wupd);
    for (cudaEvent_t e : h->ev_dw)
        if (e) cudaEventDestroy(e);
    if (h->ev_hi_join) cudaEventDestroy(h->ev_hi_join);
    if (h->h_loss) cudaFreeHost(h->h_loss);
    if (h->ev_batch) cudaEventDestroy(h->ev_batch);
    if (h->ev_step) cudaEventDestroy(h->ev_step);
    for (auto e : h->prof_pool) cudaEventDestroy(e);
    h->n_plans = 0;
    nif_free_retired(h);
    nif_field_free(h);
    if (h->d_pose_t) cudaFree(h->d_pose_t);
    delete h;
}

extern "C" const char* nif_last_error(const nif_handle* h) {
    if (!h) return g_create_err.c_str();
    return h->err.c_str();
}

// ---------------------------------------------------------------------------
// Parameters
// ---------------------------------------------------------------------------
static bool group_range(const nif_handle* h, int group, size_t* off, size_t* n) {
    if (group == NIF_PARAM_TABLES) { *off = h->off_tables; *n = (size_t)h->L * h->T * h->Fd; return true; }
    if (group == NIF_PARAM_LOGVAR) { *off = h->off_s; *n = 5; return true; }
    int l = group - NIF_PARAM_LAYER0;
    if (l >= 0 && l < h->n_layers) { *off = h->off_layer[l]; *n = (size_t)h->lay_in[l] * h->lay_out[l]; return true; }
    return false;
}

extern "C" nif_status nif_param_bytes(const nif_handle* h, int group, size_t* bytes) {
    size_t off, n;
    if (!h || !bytes || !group_range(h, group, &off, &n)) return NIF_ERR_ARG;
    *bytes = n * sizeof(float);
    return NIF_OK;
}

static nif_status copy_group(nif_handle* h, float* base, int group, void* host, size_t bytes, bool to_host) {
    size_t off, n;
    if (!h || !host || !group_range(h, group, &off, &n)) return nif_fail(h, NIF_ERR_ARG, "parameter group");
    if (bytes != n * sizeof(float)) return nif_fail(h, NIF_ERR_ARG, "parameter size mismatch");
    NIF_CK(h, cudaDeviceSynchronize());
    if (to_host) NIF_CK(h, cudaMemcpy(host, base + off, bytes, cudaMemcpyDeviceToHost));
    else NIF_CK(h, cudaMemcpy(base + off, host, bytes, cudaMemcpyHostToDevice));
    return NIF_OK;
}

extern "C" nif_status nif_get_params(nif_handle* h, int group, void* dst, size_t bytes) {
    if (!h) return NIF_ERR_ARG;
    return copy_group(h, h->d_params, group, dst, bytes, true);
}

extern "C" nif_status nif_set_params(nif_handle* h, int group, const void* src, size_t bytes) {
    if (!h) return NIF_ERR_ARG;
    nif_status st = copy_group(h, h->d_params, group, const_cast<void*>(src), bytes, false);
    h->lowp_dirty = true;
    h->x3_dirty = true;
    return st;
}

extern "C" nif_status nif_get_grad(nif_handle* h, int group, void* dst, size_t bytes) {
    if (!h) return NIF_ERR_ARG;
    return copy_group(h, h->d_grad, group, dst, bytes, true);
}

extern "C" nif_status nif_set_grad(nif_handle* h, int group, const void* src, size_t bytes) {
    if (!h) return NIF_ERR_ARG;
    return copy_group(h, h->d_grad, group, const_cast<void*>(src), bytes, false);
}

extern "C" nif_status nif_zero_grad(nif_handle* h, void* stream) {
    if (!h) return NIF_ERR_ARG;
    NIF_CK(h, cudaMemsetAsync(h->d_grad, 0, sizeof(float) * h->n_params, (cudaStream_t)stream));
    return NIF_OK;
}

extern "C" nif_status nif_reset_optimizer(nif_handle* h) {
    if (!h) return NIF_ERR_ARG;
    NIF_CK(h, cudaDeviceSynchronize());
    NIF_CK(h, cudaMemset(h->d_m, 0, sizeof(float) * h->n_params));
    NIF_CK(h, cudaMemset(h->d_v, 0, sizeof(float) * h->n_params));
    h->adam_step = 0;
    return reset_loss_scale(h);
}

extern "C" nif_status nif_adam_step_scaled(nif_handle* h, float lr_grid, float lr_mlp, void* stream) {
    if (!h) return NIF_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    nif_status st = nif_grad_check_run(h, s);
    if (st != NIF_OK) return st;
    return nif_adam_scaled_run(h, lr_grid, lr_mlp, s);
}

extern "C" nif_status nif_loss_scale(nif_handle* h, float* scale, int* skipped) {
    if (!h) return NIF_ERR_ARG;
    NifLossScale ls;
    NIF_CK(h, cudaDeviceSynchronize());
    NIF_CK(h, cudaMemcpy(&ls, h->d_ls, sizeof(ls), cudaMemcpyDeviceToHost));
    if (scale) *scale = ls.scale;
    if (skipped) *skipped = ls.skipped;
    return NIF_OK;
}

extern "C" nif_status nif_set_loss_scale(nif_handle* h, float scale) {
    if (!h) return NIF_ERR_ARG;
    if (!(scale > 0.f) || !std::isfinite(scale)) return nif_fail(h, NIF_ERR_ARG, "loss scale must be positive and finite");
    NIF_CK(h, cudaDeviceSynchronize());
    NIF_CK(h, cudaMemcpy(&h->d_ls->scale, &scale, sizeof(float), cudaMemcpyHostToDevice));
    return NIF_OK;
}

extern "C" nif_status nif_adam_step(nif_handle* h, float lr_grid, float lr_mlp, void* stream) {
    if (!h) return NIF_ERR_ARG;
    return nif_adam_run(h, lr_grid, lr_mlp, (cudaStream_t)stream);
}

// ---------------------------------------------------------------------------
// Checkpoints
// ---------------------------------------------------------------------------
namespace {

struct CkptHeader {
    char magic[8];
    uint32_t version, n_params_lo, n_params_hi, L, T, W, H, in_dim, N, P;
    int64_t adam_step;
    uint32_t pad[2];
};
static_assert(sizeof(CkptHeader) == 64, "checkpoint header is 64 bytes");

uint32_t crc32_ieee(const uint8_t* p, size_t n) {
    static uint32_t table[256];
    static bool init = false;
    if (!init) {
        for (uint32_t i = 0; i < 256; i++) {
            uint32_t c = i;
            for (int k = 0; k < 8; k++) c = (c & 1u) ? 0xEDB88320u ^ (c >> 1) : c >> 1;
            table[i] = c;
        }
        init = true;
    }
    uint32_t c = 0xFFFFFFFFu;
    for (size_t i = 0; i < n; i++) c = table[(c ^ p[i]) & 0xFFu] ^ (c >> 8);
    return c ^ 0xFFFFFFFFu;
}

CkptHeader ckpt_header(const nif_handle* h) {
    CkptHeader hd{};
    std::memcpy(hd.magic, "NIFCKPT1", 8);
    hd.version = 3;
    hd.n_params_lo = (uint32_t)(h->n_params & 0xFFFFFFFFu);
    hd.n_params_hi = (uint32_t)(h->n_params >> 32);
    hd.L = (uint32_t)h->L;
    hd.T = h->T;
    hd.W = (uint32_t)h->W;
    hd.H = (uint32_t)h->H;
    hd.in_dim = (uint32_t)h->in_dim;
    hd.N = (uint32_t)h->N;
    hd.P = (uint32_t)h->P;
    hd.adam_step = h->adam_step;
    return hd;
}

}  // namespace

// After the mixed path's state: the learned deformation field's section, a
// 16-byte header (instances, nodes per axis, Adam step count) and its values,
// first and second moments, [n][G^3] float4 each (empty without a field).
struct CkptField {
    int32_t n, G;
    int64_t step;
};
static_assert(sizeof(CkptField) == 16, "checkpoint field header is 16 bytes");
static_assert(sizeof(NifLossScale) == 40, "checkpoint mixed-precision state is 40 bytes");

static size_t ckpt_field_bytes(int64_t n, int64_t G) { return 3 * sizeof(float4) * (size_t)(n * G * G * G); }

extern "C" nif_status nif_checkpoint_bytes(const nif_handle* h, size_t* bytes) {
    if (!h || !bytes) return NIF_ERR_ARG;
    *bytes = sizeof(CkptHeader) + 3 * sizeof(float) * h->n_params + sizeof(NifLossScale) + sizeof(CkptField) +
             ckpt_field_bytes(h->field_n, h->field_G) + sizeof(uint32_t);
    return NIF_OK;
}

extern "C" nif_status nif_checkpoint_save(nif_handle* h, void* dst, size_t bytes) {
    size_t need = 0;
    if (nif_checkpoint_bytes(h, &need) != NIF_OK || !dst || bytes != need)
        return h ? nif_fail(h, NIF_ERR_ARG, "checkpoint buffer size") : NIF_ERR_ARG;
    uint8_t* o = static_cast<uint8_t*>(dst);
    CkptHeader hd = ckpt_header(h);
    std::memcpy(o, &hd, sizeof hd);
    size_t nb = sizeof(float) * h->n_params;
    NIF_CK(h, cudaDeviceSynchronize());
    NIF_CK(h, cudaMemcpy(o + sizeof hd, h->d_params, nb, cudaMemcpyDeviceToHost));
    NIF_CK(h, cudaMemcpy(o + sizeof hd + nb, h->d_m, nb, cudaMemcpyDeviceToHost));
    NIF_CK(h, cudaMemcpy(o + sizeof hd + 2 * nb, h->d_v, nb, cudaMemcpyDeviceToHost));
    NIF_CK(h, cudaMemcpy(o + sizeof hd + 3 * nb, h->d_ls, sizeof(NifLossScale), cudaMemcpyDeviceToHost));
    uint8_t* f = o + sizeof hd + 3 * nb + sizeof(NifLossScale);
    const CkptField fh{h->field_n, h->field_G, (int64_t)h->field_step};
    std::memcpy(f, &fh, sizeof fh);
    const size_t fb = ckpt_field_bytes(h->field_n, h->field_G) / 3;
    if (fb) {
        NIF_CK(h, cudaMemcpy(f + sizeof fh, h->d_field, fb, cudaMemcpyDeviceToHost));
        NIF_CK(h, cudaMemcpy(f + sizeof fh + fb, h->d_field_m, fb, cudaMemcpyDeviceToHost));
        NIF_CK(h, cudaMemcpy(f + sizeof fh + 2 * fb, h->d_field_v, fb, cudaMemcpyDeviceToHost));
    }
    const size_t body = need - sizeof(uint32_t);
    uint32_t crc = crc32_ieee(o, body);
    std::memcpy(o + body, &crc, sizeof crc);
    return NIF_OK;
}

extern "C" nif_status nif_checkpoint_load(nif_handle* h, const void* src, size_t bytes) {
    if (!h || !src) return NIF_ERR_ARG;
    const size_t nb = sizeof(float) * h->n_params;
    const size_t fpos = sizeof(CkptHeader) + 3 * nb + sizeof(NifLossScale);     // the field section
    if (bytes < fpos + sizeof(CkptField) + sizeof(uint32_t))
        return nif_fail(h, NIF_ERR_ARG, "checkpoint size does not match this configuration");
    const uint8_t* in = static_cast<const uint8_t*>(src);
    CkptHeader hd;
    std::memcpy(&hd, in, sizeof hd);
    CkptHeader mine = ckpt_header(h);
    mine.adam_step = hd.adam_step;
    if (std::memcmp(&hd, &mine, sizeof hd) != 0) return nif_fail(h, NIF_ERR_ARG, "checkpoint header mismatch");
    CkptField fh;
    std::memcpy(&fh, in + fpos, sizeof fh);
    if (!(fh.n == 0 && fh.G == 0) && !(fh.n > 0 && fh.G >= 2 && fh.G <= NIF_FIELD_MAX_G))
        return nif_fail(h, NIF_ERR_ARG, "checkpoint field section malformed");
    const size_t fb = ckpt_field_bytes(fh.n, fh.G) / 3;
    const size_t body = fpos + sizeof fh + 3 * fb;
    if (bytes != body + sizeof(uint32_t))
        return nif_fail(h, NIF_ERR_ARG, "checkpoint size does not match this configuration");
    uint32_t crc = 0;
    std::memcpy(&crc, in + body, sizeof crc);
    if (crc != crc32_ieee(in, body)) return nif_fail(h, NIF_ERR_ARG, "checkpoint CRC mismatch");
    // a query plan's graph holds the field as captured (see nif_set_field)
    if ((fh.n != h->field_n || fh.G != h->field_G) && h->n_plans > 0)
        return nif_fail(h, NIF_ERR_STATE, "destroy the query plans before loading a checkpoint with another field");
    if (fh.n > 0) {
        // allocate (or keep) a field of the checkpoint's shape, then overwrite it
        std::vector<float> zero((size_t)fh.n * fh.G * fh.G * fh.G * 3, 0.f);
        nif_status st = nif_set_field(h, fh.n, fh.G, zero.data());
        if (st != NIF_OK) return st;
        const uint8_t* f = in + fpos + sizeof fh;
        NIF_CK(h, cudaMemcpy(h->d_field, f, fb, cudaMemcpyHostToDevice));
        NIF_CK(h, cudaMemcpy(h->d_field_m, f + fb, fb, cudaMemcpyHostToDevice));
        NIF_CK(h, cudaMemcpy(h->d_field_v, f + 2 * fb, fb, cudaMemcpyHostToDevice));
        h->field_step = (long)fh.step;
    } else if (h->field_n > 0) {
        nif_status st = nif_set_field(h, 0, 0, nullptr);
        if (st != NIF_OK) return st;
    }
    NIF_CK(h, cudaDeviceSynchronize());
    NIF_CK(h, cudaMemcpy(h->d_params, in + sizeof hd, nb, cudaMemcpyHostToDevice));
    NIF_CK(h, cudaMemcpy(h->d_m, in + sizeof hd + nb, nb, cudaMemcpyHostToDevice));
    NIF_CK(h, cudaMemcpy(h->d_v, in + sizeof hd + 2 * nb, nb, cudaMemcpyHostToDevice));
    NIF_CK(h, cudaMemcpy(h->d_ls, in + sizeof hd + 3 * nb, sizeof(NifLossScale), cudaMemcpyHostToDevice));
    NIF_CK(h, cudaMemset(h->d_grad, 0, nb));
    h->adam_step = hd.adam_step;
    h->lowp_dirty = true;
    h->x3_dirty = true;
    return NIF_OK;
}

extern "C" nif_status nif_get_voxels(nif_handle* h, unsigned char* occ, int64_t* tri_ptr, int32_t* tri_idx,
                                     int64_t cap, int64_t* n_pairs) {
    if (!h || !occ) return NIF_ERR_ARG;
    int64_t nvox = (int64_t)h->N * h->N * h->N;
    NIF_CK(h, cudaDeviceSynchronize());
    NIF_CK(h, cudaMemcpy(occ, h->d_occ, nvox, cudaMemcpyDeviceToHost));
    if (n_pairs) *n_pairs = h->n_pairs;
    if (tri_ptr) {
        std::vector<uint32_t> p(nvox + 1);
        NIF_CK(h, cudaMemcpy(p.data(), h->d_tri_ptr, sizeof(uint32_t) * (nvox + 1), cudaMemcpyDeviceToHost));
        for (int64_t v = 0; v <= nvox; v++) tri_ptr[v] = p[v];
        if (tri_idx) {
            int64_t n = std::min(cap, h->n_pairs);
            if (n > 0) NIF_CK(h, cudaMemcpy(tri_idx, h->d_tri_idx, sizeof(int32_t) * n, cudaMemcpyDeviceToHost));
        }
    }
    return NIF_OK;
}

// target poses of nif_field_step into their own device array
static nif_status upload_target_poses(nif_handle* h, const nif_pose* poses, int n_inst, cudaStream_t s) {
    if (n_inst > h->inst_cap_t) {
        NIF_CK(h, cudaDeviceSynchronize());
        if (h->d_pose_t) cudaFree(h->d_pose_t);
        h->d_pose_t = nullptr;
        NIF_CK(h, cudaMalloc(&h->d_pose_t, sizeof(float4) * (size_t)n_inst));
        h->inst_cap_t = n_inst;
    }
    std::vector<float4> p(n_inst);
    for (int i = 0; i < n_inst; i++) p[i] = make_float4(NIF_KBEND * poses[i].bend, poses[i].twist, poses[i].taper, 0.f);
    NIF_CK(h, cudaMemcpyAsync(h->d_pose_t, p.data(), sizeof(float4) * n_inst, cudaMemcpyHostToDevice, s));
    NIF_CK(h, cudaStreamSynchronize(s));     // the staging vector dies with this scope
    return NIF_OK;
}

static nif_status seg_single_pass(nif_handle* h, const nif_ray* rays, const int* inst_off, int n_inst, int n_rays,
                                  uint32_t* offs, nif_segment* segs, int64_t seg_cap, bool segs_grow,
                                  int64_t* total_out, cudaStream_t s);

nif_status nif_check_status(nif_handle* h, cudaStream_t s) {
    NIF_CK(h, cudaStreamSynchronize(s));
    int st = 0;
    NIF_CK(h, cudaMemcpy(&st, h->d_status, sizeof(int), cudaMemcpyDeviceToHost));
    if (st != 0) {
        NIF_CK(h, cudaMemset(h->d_status, 0, sizeof(int)));
        return nif_fail(h, (nif_status)st, "device-side error latched by a kernel");
    }
    return NIF_OK;
}

// ---------------------------------------------------------------------------
// Stages
// ---------------------------------------------------------------------------
nif_status nif_check_inst(nif_handle* h, const nif_pose* poses, int n_inst, const int* inst_off, int n_rays) {
    if (!poses || n_inst < 1) return nif_fail(h, NIF_ERR_ARG, "poses");
    if (h->field_G > 0 && n_inst > h->field_n)
        return nif_fail(h, NIF_ERR_ARG, "more instances than the handle's field has (nif_set_field)");
    if (n_inst > 1 && !inst_off) return nif_fail(h, NIF_ERR_ARG, "inst_offsets required for n_inst > 1");
    if (n_rays < 0) return nif_fail(h, NIF_ERR_ARG, "n_rays");
    for (int i = 0; i < n_inst; i++)
        if (!(std::fabs(poses[i].bend) <= 1.0f && std::fabs(poses[i].twist) <= 4.0f && std::fabs(poses[i].taper) <= 1.0f))
            return nif_fail(h, NIF_ERR_ARG, "pose outside |bend| <= 1, |twist| <= 4, |taper| <= 1");
    return NIF_OK;
}

extern "C" nif_status nif_segments(nif_handle* h, const nif_pose* poses, int n_inst, const nif_ray* rays,
                                   const int* inst_off, int n_rays, uint32_t* ray_offsets, nif_segment* segs,
                                   int64_t seg_cap, int64_t* n_segs_host, void* stream) {
    if (!h) return NIF_ERR_ARG;
    nif_status st = nif_check_inst(h, poses, n_inst, inst_off, n_rays);
    if (st != NIF_OK) return st;
    if (!ray_offsets || (n_rays > 0 && !rays)) return nif_fail(h, NIF_ERR_ARG, "buffers");
    cudaStream_t s = (cudaStream_t)stream;
    if ((st = nif_upload_poses(h, poses, n_inst, s)) != NIF_OK) return st;
    if ((st = nif_refit_run(h, n_inst, s)) != NIF_OK) return st;
    if (segs) {
        // one traversal into scratch, then scatter into the caller's rows
        int64_t t = 0;
        if ((st = seg_single_pass(h, rays, inst_off, n_inst, n_rays, ray_offsets, segs, seg_cap, false, &t, s)) !=
            NIF_OK)
            return st;
    } else {
        if ((st = nif_grow(h, h->b_counts, sizeof(uint32_t) * ((size_t)n_rays + 1))) != NIF_OK) return st;
        uint32_t* counts = (uint32_t*)h->b_counts.p;
        if ((st = nif_seg_count_run(h, rays, inst_off, n_inst, n_rays, counts, s)) != NIF_OK) return st;
        if ((st = nif_scan_run(h, counts, ray_offsets, n_rays, s)) != NIF_OK) return st;
    }
    NIF_CK(h, cudaStreamSynchronize(s));
    uint32_t tot = 0;
    NIF_CK(h, cudaMemcpy(&tot, ray_offsets + n_rays, sizeof(uint32_t), cudaMemcpyDeviceToHost));
    if (n_segs_host) *n_segs_host = tot;
    st = nif_check_status(h, s);
    if (st != NIF_OK) return st;
    if (segs && (int64_t)tot > seg_cap) return nif_fail(h, NIF_ERR_CAPACITY, "segment capacity exceeded");
    return NIF_OK;
}

extern "C" nif_status nif_segments_walk(nif_handle* h, const nif_pose* poses, int n_inst, const nif_ray* rays,
                                        const int* inst_off, int n_rays, uint32_t* ray_offsets, nif_segment* segs,
                                        int64_t seg_cap, int64_t* n_segs_host, unsigned flags, void* stream) {
    if (!h) return NIF_ERR_ARG;
    nif_status st = nif_check_inst(h, poses, n_inst, inst_off, n_rays);
    if (st != NIF_OK) return st;
    if (!ray_offsets || (n_rays > 0 && !rays)) return nif_fail(h, NIF_ERR_ARG, "buffers");
    if (flags & ~NIF_WALK_FIRST_HIT) return nif_fail(h, NIF_ERR_ARG, "unknown walk flags");
    if ((flags & NIF_WALK_FIRST_HIT) && segs) return nif_fail(h, NIF_ERR_ARG, "NIF_WALK_FIRST_HIT counts only: segs must be NULL");
    if (h->cfg.flags & NIF_FLAG_BILINEAR_FACES)
        return nif_fail(h, NIF_ERR_ARG, "the exit-face walk is defined on the triangulated faces");
    cudaStream_t s = (cudaStream_t)stream;
    if ((st = nif_upload_poses(h, poses, n_inst, s)) != NIF_OK) return st;
    if ((st = nif_refit_run(h, n_inst, s)) != NIF_OK) return st;
    if ((st = nif_grow(h, h->b_counts, sizeof(uint32_t) * ((size_t)n_rays + 1))) != NIF_OK) return st;
    uint32_t* counts = (uint32_t*)h->b_counts.p;
    const int mode = (flags & NIF_WALK_FIRST_HIT) ? 2 : 0;
    if ((st = nif_seg_walk_run(h, rays, inst_off, n_inst, n_rays, counts, nullptr, nullptr, 0, mode, s)) != NIF_OK)
        return st;
    if ((st = nif_scan_run(h, counts, ray_offsets, n_rays, s)) != NIF_OK) return st;
    if (segs && (st = nif_seg_walk_run(h, rays, inst_off, n_inst, n_rays, nullptr, ray_offsets, segs, seg_cap, 1, s)) !=
                    NIF_OK)
        return st;
    NIF_CK(h, cudaStreamSynchronize(s));
    uint32_t tot = 0;
    NIF_CK(h, cudaMemcpy(&tot, ray_offsets + n_rays, sizeof(uint32_t), cudaMemcpyDeviceToHost));
    if (n_segs_host) *n_segs_host = tot;
    st = nif_check_status(h, s);
    if (st != NIF_OK) return st;
    if (segs && (int64_t)tot > seg_cap) return nif_fail(h, NIF_ERR_CAPACITY, "segment capacity exceeded");
    return NIF_OK;
}

extern "C" nif_status nif_linearize(nif_handle* h, const nif_pose* poses, int n_inst, const nif_ray* rays,
                                    const int* inst_off, int n_rays, const nif_segment* segs, int64_t n_segs,
                                    nif_linseg* lin, void* stream) {
    if (!h) return NIF_ERR_ARG;
    nif_status st = nif_check_inst(h, poses, n_inst, inst_off, n_rays);
    if (st != NIF_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    if ((st = nif_upload_poses(h, poses, n_inst, s)) != NIF_OK) return st;
    return nif_linearize_run(h, rays, inst_off, n_inst, segs, nullptr, n_segs, lin, s);
}

extern "C" nif_status nif_encode_points(nif_handle* h, const float* pts, int64_t n, void* feats, int out_dtype,
                                        int32_t* rows, void* stream) {
    if (!h || n < 0 || (n > 0 && (!pts || !feats))) return NIF_ERR_ARG;
    return nif_encode_points_run(h, pts, n, feats, out_dtype, rows, (cudaStream_t)stream);
}

extern "C" nif_status nif_encode_segments(nif_handle* h, const nif_linseg* lin, int64_t n, void* feats,
                                          int out_dtype, int table_dtype, void* stream) {
    if (!h || n < 0 || (n > 0 && (!lin || !feats))) return NIF_ERR_ARG;
    return nif_encode_segments_run(h, lin, nullptr, n, feats, out_dtype, table_dtype, (cudaStream_t)stream);
}

extern "C" nif_status nif_encode_points_backward(nif_handle* h, const float* pts, int64_t n, const float* dfeats,
                                                 float* dtables, float* dpts, void* stream) {
    if (!h || n < 0 || (n > 0 && (!pts || !dfeats))) return NIF_ERR_ARG;
    if (!dtables) dtables = h->d_grad + h->off_tables;
    return nif_encode_points_bwd_run(h, pts, n, dfeats, dtables, dpts, (cudaStream_t)stream);
}

extern "C" nif_status nif_pose_gradient(nif_handle* h, const nif_pose* poses, int n_inst, const int* inst_off,
                                        const nif_segment* segs, const nif_linseg* lin, int64_t n,
                                        const float* dfeats, float* dposes, float* dp_out, void* stream) {
    if (!h) return NIF_ERR_ARG;
    nif_status st = nif_check_inst(h, poses, n_inst, inst_off, 0);
    if (st != NIF_OK) return st;
    if (n < 0 || (n > 0 && (!segs || !lin || !dfeats || !dposes))) return nif_fail(h, NIF_ERR_ARG, "buffers");
    cudaStream_t s = (cudaStream_t)stream;
    if ((st = nif_upload_poses(h, poses, n_inst, s)) != NIF_OK) return st;
    float* dp = dp_out;
    if (!dp) {
        if ((st = nif_grow(h, h->b_dx, sizeof(float) * 6 * (size_t)std::max<int64_t>(n, 1))) != NIF_OK) return st;
        dp = (float*)h->b_dx.p;
    }
    if ((st = nif_encode_segments_dp_run(h, lin, nullptr, n, dfeats, dp, s)) != NIF_OK) return st;
    return nif_pose_grad_run(h, segs, lin, dp, nullptr, n, inst_off, n_inst, dposes, s);
}

extern "C" nif_status nif_encode_segments_backward(nif_handle* h, const nif_linseg* lin, int64_t n,
                                                   const float* dfeats, float* dtables, void* stream) {
    if (!h || n < 0 || (n > 0 && (!lin || !dfeats || !dtables))) return NIF_ERR_ARG;
    return nif_encode_segments_bwd_run(h, lin, nullptr, n, dfeats, dtables, (cudaStream_t)stream);
}

extern "C" nif_status nif_mlp_forward(nif_handle* h, const void* x, int x_dtype, int64_t n, float* out,
                                      int precision, float* acts, void* stream) {
    if (!h || n < 0 || (n > 0 && (!x || !out))) return NIF_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    if (precision == NIF_FP32) {
        if (x_dtype != NIF_FP32) return nif_fail(h, NIF_ERR_ARG, "FP32 MLP needs FP32 input");
        nif_status st = NIF_OK;
        float* a = acts;
        if (!a) {
            if ((st = nif_grow(h, h->b_acts, sizeof(float) * (size_t)std::max<int64_t>(n, 1) * h->W * h->H)) != NIF_OK)
                return st;
            a = (float*)h->b_acts.p;
        }
        return nif_mlp_fwd_fp32_run(h, (const float*)x, nullptr, n, out, a, s);
    }
    if (precision != x_dtype) return nif_fail(h, NIF_ERR_ARG, "tensor-core MLP input dtype must equal precision");
    return nif_mlp_fwd_tc_run(h, x, precision, nullptr, n, out, s);
}

extern "C" nif_status nif_mlp_backward(nif_handle* h, const float* x, int64_t n, const float* acts, const float* dout,
                                       float* dx, void* stream) {
    if (!h || n < 0 || (n > 0 && (!x || !acts || !dout))) return NIF_ERR_ARG;
    return nif_mlp_bwd_fp32_run(h, x, nullptr, n, acts, dout, dx, (cudaStream_t)stream);
}

// 16-bit activations and output gradients of the mixed path: [layers][n_pad][kLd]
static constexpr int kLd = 64;

static int64_t pad128(int64_t n) { return (n + 127) / 128 * 128; }

static nif_status check_mixed(nif_handle* h) {
    if (h->cfg.precision != NIF_BF16 && h->cfg.precision != NIF_FP16)
        return nif_fail(h, NIF_ERR_ARG, "mixed-precision training needs a BF16 or FP16 handle");
    if (h->W != 32 && h->W != 64) return nif_fail(h, NIF_ERR_ARG, "mixed-precision training needs W = 32 or 64");
    if (h->in_dim % 16 != 0) return nif_fail(h, NIF_ERR_ARG, "mixed-precision training needs in_dim % 16 == 0");
    return NIF_OK;
}

extern "C" nif_status nif_mlp_backward_lowp(nif_handle* h, const void* x, int x_dtype, int64_t n, const float* dout,
                                            float* dx, void* stream) {
    if (!h || n < 0 || (n > 0 && (!x || !dout))) return NIF_ERR_ARG;
    nif_status st = check_mixed(h);
    if (st != NIF_OK) return st;
    if (x_dtype != h->cfg.precision) return nif_fail(h, NIF_ERR_ARG, "x_dtype must equal the handle's precision");
    if ((reinterpret_cast<uintptr_t>(x) & 15) != 0) return nif_fail(h, NIF_ERR_ARG, "x not 16-byte aligned");
    if (n == 0) return NIF_OK;
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t np = pad128(n);
    if ((st = nif_grow(h, h->b_acts, 2 * (size_t)np * kLd * h->H)) != NIF_OK) return st;
    if ((st = nif_grow(h, h->b_dys, 2 * (size_t)np * kLd * (h->H + 1))) != NIF_OK) return st;
    if ((st = nif_grow(h, h->b_out, sizeof(float) * NIF_OUT * (size_t)np)) != NIF_OK) return st;
    if (!dx) {
        if ((st = nif_grow(h, h->b_dx, sizeof(float) * (size_t)h->in_dim * n)) != NIF_OK) return st;
        dx = (float*)h->b_dx.p;
    }
    uint16_t* acts = (uint16_t*)h->b_acts.p;
    uint16_t* dys = (uint16_t*)h->b_dys.p;
    // activations recomputed from x with the current weights
    if ((st = nif_mlp_fwd_tc_acts_run(h, x, x_dtype, nullptr, n, (float*)h->b_out.p, acts, np, kLd, s)) != NIF_OK)
        return st;
    if ((st = nif_mlp_bwd_tc_run(h, dout, acts, nullptr, n, np, kLd, dys, dx, s)) != NIF_OK) return st;
    return nif_mlp_dw_tc_run(h, x, acts, dys, nullptr, n, np, kLd, s);
}

extern "C" nif_status nif_labels(nif_handle* h, const nif_segment* segs, const nif_linseg* lin, int64_t n,
                                 nif_label* labels, void* stream) {
    if (!h || n < 0 || (n > 0 && (!segs || !lin || !labels))) return NIF_ERR_ARG;
    return nif_labels_run(h, segs, lin, nullptr, n, labels, (cudaStream_t)stream);
}

extern "C" nif_status nif_loss(nif_handle* h, const float* out, const nif_label* labels, const nif_linseg* lin,
                               int64_t n, float* dout, double* parts_host, void* stream) {
    if (!h || n < 0 || (n > 0 && (!out || !labels || !lin))) return NIF_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    // hit count of these labels (the label stage counted its own batch; recount here)
    nif_status st = nif_labels_count_hits(h, labels, n, s);
    if (st != NIF_OK) return st;
    if ((st = nif_loss_run(h, out, labels, lin, nullptr, n, dout, s)) != NIF_OK) return st;
    if (parts_host) {
        double acc[16];
        NIF_CK(h, cudaStreamSynchronize(s));
        NIF_CK(h, cudaMemcpy(acc, h->d_lossacc, sizeof(acc), cudaMemcpyDeviceToHost));
        parts_host[0] = acc[8];
        for (int i = 0; i < 5; i++) parts_host[1 + i] = acc[9 + i];
    }
    return NIF_OK;
}

extern "C" nif_status nif_reconstruct(nif_handle* h, const nif_pose* poses, int n_inst, const nif_ray* rays,
                                      const int* inst_off, int n_rays, const uint32_t* ray_offsets,
                                      const nif_segment* segs, const nif_linseg* lin, const float* out,
                                      nif_hit* hits, unsigned flags, void* stream) {
    if (!h) return NIF_ERR_ARG;
    nif_status st = nif_check_inst(h, poses, n_inst, inst_off, n_rays);
    if (st != NIF_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    if ((st = nif_upload_poses(h, poses, n_inst, s)) != NIF_OK) return st;
    return nif_reconstruct_run(h, rays, inst_off, n_inst, n_rays, ray_offsets, segs, INT64_MAX, lin, out, hits, flags,
                               s);
}

extern "C" nif_status nif_sample_rays(nif_handle* h, unsigned long long seed, int stream_id, int n, nif_ray* rays,
                                      void* stream) {
    if (!h || n < 0 || (n > 0 && !rays)) return NIF_ERR_ARG;
    return nif_sample_rays_run(h, seed, stream_id, n, rays, (cudaStream_t)stream);
}

// ---------------------------------------------------------------------------
// Whole paths
// ---------------------------------------------------------------------------

// Single traversal (counts + ray-unordered segments into handle scratch),
// scan, then scatter into the CSR rows `offs` / `segs` (capacity seg_cap,
// or sized to the total when segs_grow is set). Blocks the host once to read
// the total. Falls back to a second traversal when the scratch was short.
static nif_status seg_single_pass(nif_handle* h, const nif_ray* rays, const int* inst_off, int n_inst, int n_rays,
                                  uint32_t* offs, nif_segment* segs, int64_t seg_cap, bool segs_grow,
                                  int64_t* total_out, cudaStream_t s) {
    nif_status st;
    if ((st = nif_grow(h, h->b_counts, sizeof(uint32_t) * ((size_t)n_rays + 1))) != NIF_OK) return st;
    uint32_t* counts = (uint32_t*)h->b_counts.p;
    double hint = h->query_seg_per_ray > 0.0 ? h->query_seg_per_ray * 1.25 + 0.5 : 8.0;
    int64_t tcap = std::max<int64_t>(4096, (int64_t)(hint * h->seg_scratch_scale * (double)n_rays));
    if ((st = nif_grow(h, h->b_temp, sizeof(nif_segment) * (size_t)tcap)) != NIF_OK) return st;
    // the whole buffer, unless the scratch knob asks for less
    if (h->seg_scratch_scale >= 1.0) tcap = (int64_t)(h->b_temp.bytes / sizeof(nif_segment));
    uint32_t* cursor = reinterpret_cast<uint32_t*>(h->d_count + 1);
    NIF_CK(h, cudaMemsetAsync(cursor, 0, sizeof(uint32_t), s));
    if ((st = nif_seg_temp_run(h, rays, inst_off, n_inst, n_rays, counts, (nif_segment*)h->b_temp.p, tcap, cursor, s)) !=
        NIF_OK)
        return st;
    if ((st = nif_scan_run(h, counts, offs, n_rays, s)) != NIF_OK) return st;
    NIF_CK(h, cudaMemcpyAsync(h->h_pinned, offs + n_rays, sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
    NIF_CK(h, cudaStreamSynchronize(s));
    int64_t total = (uint32_t)h->h_pinned[0];
    *total_out = total;
    if (n_rays > 0) h->query_seg_per_ray = (double)total / n_rays;
    if (segs_grow) {
        if ((st = nif_grow(h, h->b_segs, sizeof(nif_segment) * (size_t)std::max<int64_t>(total, 1))) != NIF_OK)
            return st;
        segs = (nif_segment*)h->b_segs.p;
        seg_cap = total;
    }
    if (!segs) return NIF_OK;
    if (total <= tcap) {
        NIF_CK(h, cudaMemsetAsync(counts, 0, sizeof(uint32_t) * (size_t)n_rays, s));
        return nif_seg_scatter_run(h, (const nif_segment*)h->b_temp.p, cursor, total, offs, counts, n_rays, segs,
                                   seg_cap, s);
    }
    return nif_seg_emit_run(h, rays, inst_off, n_inst, n_rays, offs, segs, seg_cap, s);
}

// segments of the caller's rays into the handle's scratch; returns the device
// pointer of the clamped total (<= cap)
static nif_status segment_into_scratch(nif_handle* h, const nif_pose* poses, int n_inst, const nif_ray* rays,
                                       const int* inst_off, int n_rays, int64_t cap, bool host_total,
                                       int64_t* total_host, cudaStream_t s, bool latch = false) {
    nif_status st;
    if ((st = nif_upload_poses(h, poses, n_inst, s)) != NIF_OK) return st;
    if ((st = nif_refit_run(h, n_inst, s)) != NIF_OK) return st;
    if ((st = nif_grow(h, h->b_counts, sizeof(uint32_t) * ((size_t)n_rays + 1))) != NIF_OK) return st;
    if ((st = nif_grow(h, h->b_offsets, sizeof(uint32_t) * ((size_t)n_rays + 2))) != NIF_OK) return st;
    uint32_t* counts = (uint32_t*)h->b_counts.p;
    uint32_t* offs = (uint32_t*)h->b_offsets.p;
    if (host_total) {
        int64_t tot = 0;
        if ((st = seg_single_pass(h, rays, inst_off, n_inst, n_rays, offs, nullptr, 0, true, &tot, s)) != NIF_OK)
            return st;
        *total_host = tot;
        if (cap < 0) cap = tot;
    } else {
        // a batch of at most `cap` segments of whole rays, with no host round
        // trip: one traversal into scratch in warp order, CSR offsets, scatter
        // into ray order and per-row sort; should the scratch overflow, a
        // second traversal (device-gated) writes the rows directly
        int64_t tcap = (int64_t)(2.0 * h->seg_scratch_scale * (double)cap) + 4096;
        if ((st = nif_grow(h, h->b_temp, sizeof(nif_segment) * (size_t)tcap)) != NIF_OK) return st;
        if (h->seg_scratch_scale >= 1.0) tcap = (int64_t)(h->b_temp.bytes / sizeof(nif_segment));
        if ((st = nif_grow(h, h->b_segs, sizeof(nif_segment) * (size_t)std::max<int64_t>(cap, 1))) != NIF_OK)
            return st;
        nif_segment* segs = (nif_segment*)h->b_segs.p;
        uint32_t* cursor = reinterpret_cast<uint32_t*>(h->d_count + 1);
        NIF_CK(h, cudaMemsetAsync(cursor, 0, sizeof(uint32_t), s));
        if ((st = nif_seg_temp_run(h, rays, inst_off, n_inst, n_rays, counts, (nif_segment*)h->b_temp.p, tcap,
                                   cursor, s)) != NIF_OK)
            return st;
        if ((st = nif_scan_run(h, counts, offs, n_rays, s)) != NIF_OK) return st;
        NIF_CK(h, cudaMemsetAsync(counts, 0, sizeof(uint32_t) * (size_t)n_rays, s));
        if ((st = nif_seg_scatter_run(h, (const nif_segment*)h->b_temp.p, cursor, tcap, offs, counts, n_rays, segs,
                                      cap, s)) != NIF_OK)
            return st;
        if ((st = nif_seg_emit_if_overflow_run(h, rays, inst_off, n_inst, n_rays, offs, segs, cap, cursor, tcap, s)) !=
            NIF_OK)
            return st;
        // only complete rows: the row that crosses `cap` holds an arbitrary
        // subset of its ray's segments (latch: that is an error, not the end
        // of a training batch)
        return nif_clamp_count_run(h, offs, n_rays, cap, offs + n_rays + 1, latch, s, true);
    }
    // clamped count lives right after the offsets
    return nif_clamp_count_run(h, offs, n_rays, cap, offs + n_rays + 1, host_total, s);
}

// The query's encoding and MLP as two kernels per chunk (FP32, or a handle
// the fused kernel does not cover): features of a chunk go through a buffer.
static nif_status query_encode_mlp(nif_handle* h, const nif_linseg* lin, const uint32_t* n_dev, int64_t cap,
                                   int n_rays, float* out, cudaStream_t s) {
    nif_status st;
    const int prec = h->cfg.precision;
    const size_t esz = prec == NIF_FP32 ? 4 : 2;
    // encode + MLP in chunks with device-side counts: FP32 chunks stay
    // resident in L2 between the two kernels; the tensor-core MLP is a
    // persistent kernel whose pipeline needs many tiles per CTA
    const int64_t chunk = std::min<int64_t>(h->tune.tc_chunk, cap);
    const int n_chunks = (int)((cap + chunk - 1) / chunk);
    if ((st = nif_grow(h, h->b_feat, esz * (size_t)h->in_dim * chunk)) != NIF_OK) return st;
    if (prec == NIF_FP32 && (st = nif_grow(h, h->b_acts, sizeof(float) * (size_t)chunk * h->W * h->H)) != NIF_OK)
        return st;
    if (n_chunks > h->chunk_counts_cap) {
        NIF_CK(h, cudaDeviceSynchronize());
        if (h->d_chunk_counts) cudaFree(h->d_chunk_counts);
        h->d_chunk_counts = nullptr;
        h->chunk_counts_cap = 0;
        NIF_CK(h, cudaMalloc(&h->d_chunk_counts, sizeof(uint32_t) * (size_t)n_chunks));
        h->chunk_counts_cap = n_chunks;
    }
    if ((st = nif_chunk_counts_run(h, n_dev, chunk, n_chunks, h->d_chunk_counts, s)) != NIF_OK) return st;
    // chunks past the segments the last query found (+2 %) are expected to be
    // empty: they skip the distinct-point list, whose preparation would cost
    // the full chunk size even for a zero count (encoded correctly either way)
    const int n_expected = h->q_hint > 0.0
                               ? (int)std::min<int64_t>(n_chunks, (int64_t)std::ceil(h->q_hint * 1.02 * n_rays / chunk))
                               : n_chunks;
    for (int c = 0; c < n_chunks; c++) {
        const int64_t c0 = (int64_t)c * chunk;
        const int64_t len = std::min(chunk, cap - c0);
        const uint32_t* cn = h->d_chunk_counts + c;
        const bool dedup = c < n_expected;
        if (prec == NIF_FP32) {
            if ((st = nif_encode_segments_run(h, lin + c0, cn, len, h->b_feat.p, NIF_FP32, NIF_FP32, s, false, dedup)) !=
                NIF_OK)
                return st;
            if ((st = nif_mlp_fwd_fp32_run(h, (const float*)h->b_feat.p, cn, len, out + c0 * NIF_OUT,
                                           (float*)h->b_acts.p, s, 0, true)) != NIF_OK)
                return st;
        } else {
            if ((st = nif_encode_segments_run(h, lin + c0, cn, len, h->b_feat.p, prec, NIF_FP16, s, false, dedup)) !=
                NIF_OK)
                return st;
            if ((st = nif_mlp_fwd_tc_run(h, h->b_feat.p, prec, cn, len, out + c0 * NIF_OUT, s)) != NIF_OK) return st;
        }
    }
    return NIF_OK;
}

extern "C" nif_status nif_query(nif_handle* h, const nif_pose* poses, int n_inst, const nif_ray* rays,
                                const int* inst_off, int n_rays, nif_hit* hits, unsigned flags, void* stream) {
    if (!h) return NIF_ERR_ARG;
    nif_status st = nif_check_inst(h, poses, n_inst, inst_off, n_rays);
    if (st != NIF_OK) return st;
    if (n_rays == 0) return NIF_OK;
    if (!rays || !hits) return nif_fail(h, NIF_ERR_ARG, "rays / hits");
    cudaStream_t s = (cudaStream_t)stream;
    // capacity: segments per ray of the last query whose total has come back
    // (1.5 x, read without waiting), or the initial estimate
    if (h->q_pending && cudaEventQuery(h->ev_qtotal) == cudaSuccess) {
        h->q_hint = (double)h->h_qtotal[0] / (double)std::max(h->q_rays, 1);
        h->q_pending = false;
    }
    const double spr = h->q_hint > 0.0 ? h->q_hint * 1.5 + 0.25 : h->q_init;
    const int64_t cap = std::max<int64_t>(4096, (int64_t)std::ceil(spr * (double)n_rays));
    // segments of whole rays within the capacity, counts on the device; more
    // latches NIF_ERR_CAPACITY (the rays that did not fit report no hit)
    if ((st = segment_into_scratch(h, poses, n_inst, rays, inst_off, n_rays, cap, false, nullptr, s, true)) != NIF_OK)
        return st;
    uint32_t* offs = (uint32_t*)h->b_offsets.p;
    const uint32_t* n_dev = offs + n_rays + 1;
    if ((st = nif_grow(h, h->b_lin, sizeof(nif_linseg) * cap)) != NIF_OK) return st;
    if ((st = nif_grow(h, h->b_out, sizeof(float) * NIF_OUT * cap)) != NIF_OK) return st;
    nif_segment* segs = (nif_segment*)h->b_segs.p;
    nif_linseg* lin = (nif_linseg*)h->b_lin.p;
    float* out = (float*)h->b_out.p;
    if ((st = nif_linearize_run(h, rays, inst_off, n_inst, segs, n_dev, cap, lin, s)) != NIF_OK) return st;
    const int prec = h->cfg.precision;
    if (prec != NIF_FP32 && nif_mlp_enc_fusable(h)) {
        // encoding and MLP in one launch over every segment: no feature matrix
        if ((st = nif_mlp_enc_tc_run(h, lin, n_dev, cap, out, s)) != NIF_OK) return st;
    } else if ((st = query_encode_mlp(h, lin, n_dev, cap, n_rays, out, s)) != NIF_OK) {
        return st;
    }
    if ((st = nif_reconstruct_run(h, rays, inst_off, n_inst, n_rays, offs, segs, cap, lin, out, hits, flags, s,
                                  n_dev)) != NIF_OK)
        return st;
    // this call's total, for the capacity of the next ones
    NIF_CK(h, cudaMemcpyAsync(h->h_qtotal, offs + n_rays, sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
    NIF_CK(h, cudaEventRecord(h->ev_qtotal, s));
    h->q_pending = true;
    h->q_rays = n_rays;
    return NIF_OK;
}

// The error a kernel latched on the device (a non-finite loss, a timed-out
// wait), cleared once read; the caller has synchronised the work it checks.
static nif_status latched_status(nif_handle* h) {
    int dst = 0;
    NIF_CK(h, cudaMemcpy(&dst, h->d_status, sizeof(int), cudaMemcpyDeviceToHost));
    if (dst == 0) return NIF_OK;
    cudaMemset(h->d_status, 0, sizeof(int));
    return nif_fail(h, (nif_status)dst, dst == NIF_ERR_NAN ? "non-finite loss" : "device-side error latched by a kernel");
}

// The batch of one training step: segments of whole rays (at most n_segments,
// in ray order), their linearization and labels, into the handle's batch
// buffers; the hit count goes to *n_hit (device).
static nif_status train_batch(nif_handle* h, const nif_pose* poses, int n_inst, const nif_ray* rays,
                              const int* inst_off, int n_rays, int64_t n_segments, int* n_hit, cudaStream_t s) {
    nif_status st;
    // the point list of the set's previous batch names the same buffers: drop it
    h->enc_points = nif_handle::PointList{};
    if ((st = segment_into_scratch(h, poses, n_inst, rays, inst_off, n_rays, n_segments, false, nullptr, s)) != NIF_OK)
        return st;
    uint32_t* offs = (uint32_t*)h->b_offsets.p;
    const uint32_t* n_dev = offs + n_rays + 1;
    const int64_t n = n_segments;
    if ((st = nif_grow(h, h->b_lin, sizeof(nif_linseg) * n)) != NIF_OK) return st;
    if ((st = nif_grow(h, h->b_labels, sizeof(nif_label) * n)) != NIF_OK) return st;
    nif_segment* segs = (nif_segment*)h->b_segs.p;
    nif_linseg* lin = (nif_linseg*)h->b_lin.p;
    if ((st = nif_linearize_run(h, rays, inst_off, n_inst, segs, n_dev, n, lin, s)) != NIF_OK) return st;
    if ((st = nif_labels_run(h, segs, lin, n_dev, n, (nif_label*)h->b_labels.p, s, n_hit)) != NIF_OK) return st;
    // FP32 path: the distinct end points that the step's encodings (forward
    // and backward) walk are listed with the batch, off the step's stream
    // when the batch is built beside the previous step (step 3.08 -> 3.06 ms).
    // The mixed path lists them in its forward: its batch runs beside the
    // step's forward, and the longer batch cost more there (2.40 vs 2.47 ms).
    if (h->cfg.flags & NIF_FLAG_MIXED_TRAINING) return NIF_OK;
    return nif_encode_points_prepare(h, lin, n_dev, n, NIF_FP32, s);
}

// Forward, losses, backward and optimizer step on the batch in the handle's
// batch buffers (n_rays rays, at most n_segments segments; hit count *n_hit).
// ev_next (nullable) is recorded on s where the next batch may start beside
// the step: after the encoding forward (FP32 path only).
// CTAs of a training step's persistent MLP forward while the next batch is
// built beside it (NIF_KNOB_STEP_FWD_CTAS); 0 = one per SM. By default the
// FP32 forward takes three quarters of the SMs, then the fewest CTAs that give
// each the same number of 128-row tiles, and the batch's kernels keep the
// other SMs (measured on the 64^3 FP32 step: 2.97 ms on 103-114 CTAs,
// 3.01-3.04 ms on 96 or 120-152); the 16-bit forward keeps every SM (its
// step: 2.390-2.393 ms, against 2.398-2.400 ms on three quarters).
static int step_fwd_ctas(const nif_handle* h, int64_t n, bool fp32) {
    const int k = h->tune.step_fwd_ctas;
    if (k != 0) return k < 0 ? 0 : k;
    if (!fp32) return 0;
    const int64_t tiles = std::max<int64_t>((n + 127) / 128, 1);
    const int64_t c = std::max(1, h->num_sms * 3 / 4);
    const int64_t per = (tiles + c - 1) / c;
    return (int)((tiles + per - 1) / per);
}

static nif_status train_compute_on(nif_handle* h, int n_rays, int64_t n_segments, const int* n_hit, float lr_grid,
                                   float lr_mlp, double* loss_host, cudaStream_t s, cudaEvent_t ev_next,
                                   bool join_weights, int set);

// One step's forward, losses, backward and update. A step that fails before
// its update (an allocation, an argument of a stage) may have added part of
// its gradients: they are cleared, after the device has finished what was
// enqueued, so that the trainable state is the one before the step.
static nif_status train_compute(nif_handle* h, int n_rays, int64_t n_segments, const int* n_hit, float lr_grid,
                                float lr_mlp, double* loss_host, cudaStream_t s, cudaEvent_t ev_next = nullptr,
                                bool join_weights = true, int set = -1) {
    const nif_status st =
        train_compute_on(h, n_rays, n_segments, n_hit, lr_grid, lr_mlp, loss_host, s, ev_next, join_weights, set);
    if (st == NIF_OK || st == NIF_ERR_NAN || st == NIF_ERR_TIMEOUT || st == NIF_ERR_CAPACITY) return st;
    if (cudaDeviceSynchronize() == cudaSuccess && cudaMemset(h->d_grad, 0, sizeof(float) * h->n_params) == cudaSuccess)
        h->wupd_pending = false;
    else
        cudaGetLastError();
    return st;
}

static nif_status train_compute_on(nif_handle* h, int n_rays, int64_t n_segments, const int* n_hit, float lr_grid,
                                   float lr_mlp, double* loss_host, cudaStream_t s, cudaEvent_t ev_next,
                                   bool join_weights, int set) {
    nif_status st;
    const bool mixed = (h->cfg.flags & NIF_FLAG_MIXED_TRAINING) != 0;
    uint32_t* offs = (uint32_t*)h->b_offsets.p;
    const uint32_t* n_dev = offs + n_rays + 1;
    const int64_t n = n_segments;
    if ((st = nif_grow(h, h->b_feat, sizeof(float) * (size_t)h->in_dim * n)) != NIF_OK) return st;
    if ((st = nif_grow(h, h->b_dx, sizeof(float) * (size_t)h->in_dim * n)) != NIF_OK) return st;
    if ((st = nif_grow(h, h->b_out, sizeof(float) * NIF_OUT * n)) != NIF_OK) return st;
    if ((st = nif_grow(h, h->b_feat2, sizeof(float) * NIF_OUT * n)) != NIF_OK) return st;
    const int64_t np = pad128(n);
    if ((st = nif_grow(h, h->b_acts, mixed ? 2 * (size_t)np * kLd * h->H : sizeof(float) * (size_t)n * h->W * h->H)) !=
        NIF_OK)
        return st;
    if (mixed) {
        if ((st = nif_grow(h, h->b_feat, 2 * (size_t)h->in_dim * np)) != NIF_OK) return st;
        if ((st = nif_grow(h, h->b_dys, 2 * (size_t)np * kLd * (h->H + 1))) != NIF_OK) return st;
    }
    nif_linseg* lin = (nif_linseg*)h->b_lin.p;
    nif_label* lab = (nif_label*)h->b_labels.p;
    float* feat = (float*)h->b_feat.p;
    float* dx = (float*)h->b_dx.p;
    float* out = (float*)h->b_out.p;
    float* dout = (float*)h->b_feat2.p;
    float* acts = (float*)h->b_acts.p;
    if (mixed) {
        // 16-bit features from the FP16 table copy, tensor-core MLP forward
        // keeping its activations, loss on FP32 outputs, scaled tensor-core
        // backward and weight gradients, FP32 table gradients, checked Adam
        const int prec = h->cfg.precision;
        uint16_t* acts16 = (uint16_t*)h->b_acts.p;
        uint16_t* dys = (uint16_t*)h->b_dys.p;
        if ((st = nif_encode_segments_run(h, lin, n_dev, n, feat, prec, NIF_FP16, s, true)) != NIF_OK) return st;
        if ((st = nif_mlp_fwd_tc_acts_run(h, feat, prec, n_dev, n, out, acts16, np, kLd, s,
                                          h->batch_beside ? step_fwd_ctas(h, n, false) : 0)) != NIF_OK)
            return st;
        if ((st = nif_loss_run(h, out, lab, lin, n_dev, n, dout, s, true, n_hit)) != NIF_OK) return st;
        if ((st = nif_mlp_bwd_tc_run(h, dout, acts16, n_dev, n, np, kLd, dys, dx, s)) != NIF_OK) return st;
        // weight gradients on the second stream, beside the encoding backward
        NIF_CK(h, cudaEventRecord(h->ev_fork, s));
        NIF_CK(h, cudaStreamWaitEvent(h->aux, h->ev_fork, 0));
        if ((st = nif_mlp_dw_tc_run(h, feat, acts16, dys, n_dev, n, np, kLd, h->aux)) != NIF_OK) return st;
        NIF_CK(h, cudaEventRecord(h->ev_join, h->aux));
        if ((st = nif_encode_segments_bwd_run(h, lin, n_dev, n, dx, h->d_grad + h->off_tables, s, true)) != NIF_OK)
            return st;
        NIF_CK(h, cudaStreamWaitEvent(s, h->ev_join, 0));
        if ((st = nif_grad_check_run(h, s)) != NIF_OK) return st;
        if ((st = nif_adam_scaled_run(h, lr_grid, lr_mlp, s)) != NIF_OK) return st;
    } else {
        // With the weight update deferred, the weights' Adam of this step runs
        // on the second stream after its weight gradients, beside the next
        // step's encoding forward, which therefore writes the other feature
        // buffer; the next step's MLP forward waits for that update.
        const bool defer = h->tune.defer_wupd != 0;
        if (defer) {
            if ((st = nif_grow(h, h->b_feat_alt, sizeof(float) * (size_t)h->in_dim * n)) != NIF_OK) return st;
            if (h->feat_flip) feat = (float*)h->b_feat_alt.p;
            h->feat_flip ^= 1;
        }
        // the next batch may start where the handle's placement knob says
        const int at = h->tune.batch_at;
        if (ev_next && at == 0) NIF_CK(h, cudaEventRecord(ev_next, s));
        if ((st = nif_encode_segments_run(h, lin, n_dev, n, feat, NIF_FP32, NIF_FP32, s, true)) != NIF_OK) return st;
        if (ev_next && at == 1) NIF_CK(h, cudaEventRecord(ev_next, s));
        if (h->wupd_pending) {                  // the previous step's weights are updated
            NIF_CK(h, cudaStreamWaitEvent(s, h->ev_wupd, 0));
            h->wupd_pending = false;
        }
        const bool beside = h->batch_beside && at <= 1;   // the next batch starts before this forward
        if ((st = nif_mlp_fwd_fp32_run(h, feat, n_dev, n, out, acts, s, beside ? step_fwd_ctas(h, n, true) : 0)) != NIF_OK)
            return st;
        if (ev_next && at == 2) NIF_CK(h, cudaEventRecord(ev_next, s));
        if ((st = nif_loss_run(h, out, lab, lin, n_dev, n, dout, s, true, n_hit)) != NIF_OK) return st;
        // weight gradients on the second stream, beside dX_0 and the encoding backward
        if ((st = nif_mlp_bwd_fp32_run(h, feat, n_dev, n, acts, dout, dx, s, true, h->aux)) != NIF_OK) return st;
        if (ev_next && at >= 3) NIF_CK(h, cudaEventRecord(ev_next, s));
        // the encoding backward leaves some SMs to the weight gradients
        // (NIF_KNOB_STEP_BWD_CTAS; measured on the 64^3 step: 2.91-2.92 ms on
        // 128-136 of 152 SMs, 2.97 ms on all, 2.94-2.95 ms on 124 or 144)
        const int kb = h->tune.step_bwd_ctas;
        const int bwd_ctas = kb < 0 ? 0 : (kb > 0 ? kb : std::max(1, h->num_sms * 7 / 8));
        if ((st = nif_encode_segments_bwd_run(h, lin, n_dev, n, dx, h->d_grad + h->off_tables, s, true, bwd_ctas)) !=
            NIF_OK)
            return st;
        bool split = false;
        if (defer && (st = nif_adam_split_run(h, lr_grid, lr_mlp, s, h->aux, &split)) != NIF_OK) return st;
        if (split) {
            NIF_CK(h, cudaEventRecord(h->ev_wupd, h->aux));
            // a later batch built into this step's buffer set (its segment
            // count is read by the weight gradients) waits for them
            if (set >= 0) NIF_CK(h, cudaEventRecord(h->ev_dw[set], h->aux));
            h->wupd_pending = true;
            if (join_weights) {
                NIF_CK(h, cudaStreamWaitEvent(s, h->ev_wupd, 0));
                h->wupd_pending = false;
            }
        } else {
            NIF_CK(h, cudaStreamWaitEvent(s, h->ev_join, 0));
            if ((st = nif_adam_run(h, lr_grid, lr_mlp, s)) != NIF_OK) return st;
        }
    }
    if (loss_host) {
        double acc[16];
        NIF_CK(h, cudaStreamSynchronize(s));
        NIF_CK(h, cudaMemcpy(acc, h->d_lossacc, sizeof(acc), cudaMemcpyDeviceToHost));
        loss_host[0] = acc[8];
        for (int i = 0; i < 5; i++) loss_host[1 + i] = acc[9 + i];
        return latched_status(h);
    }
    return NIF_OK;
}

extern "C" nif_status nif_train_step_rays(nif_handle* h, const nif_pose* poses, int n_inst, const nif_ray* rays,
                                          const int* inst_off, int n_rays, int64_t n_segments, float lr_grid,
                                          float lr_mlp, double* loss_host, void* stream) {
    if (!h) return NIF_ERR_ARG;
    nif_status st = nif_check_inst(h, poses, n_inst, inst_off, n_rays);
    if (st != NIF_OK) return st;
    if (n_segments < 1 || !rays) return nif_fail(h, NIF_ERR_ARG, "n_segments / rays");
    const bool mixed = (h->cfg.flags & NIF_FLAG_MIXED_TRAINING) != 0;
    if (mixed && (st = check_mixed(h)) != NIF_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    if ((st = train_batch(h, poses, n_inst, rays, inst_off, n_rays, n_segments, h->d_count, s)) != NIF_OK) return st;
    return train_compute(h, n_rays, n_segments, h->d_count, lr_grid, lr_mlp, loss_host, s);
}

extern "C" nif_status nif_pose_step(nif_handle* h, const nif_pose* poses, int n_inst, const nif_ray* rays,
                                    const int* inst_off, int n_rays, int64_t n_segments, float* dposes,
                                    double* loss_host, void* stream) {
    if (!h) return NIF_ERR_ARG;
    nif_status st = nif_check_inst(h, poses, n_inst, inst_off, n_rays);
    if (st != NIF_OK) return st;
    if (n_segments < 1 || !rays || !dposes) return nif_fail(h, NIF_ERR_ARG, "n_segments / rays / dposes");
    const int prec = h->cfg.precision;
    if (prec != NIF_FP32 && (st = check_mixed(h)) != NIF_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    if ((st = segment_into_scratch(h, poses, n_inst, rays, inst_off, n_rays, n_segments, false, nullptr, s)) != NIF_OK)
        return st;
    uint32_t* offs = (uint32_t*)h->b_offsets.p;
    const uint32_t* n_dev = offs + n_rays + 1;
    const int64_t n = n_segments, np = pad128(n);
    const size_t esz = prec == NIF_FP32 ? 4 : 2;
    if ((st = nif_grow(h, h->b_lin, sizeof(nif_linseg) * n)) != NIF_OK) return st;
    if ((st = nif_grow(h, h->b_labels, sizeof(nif_label) * n)) != NIF_OK) return st;
    if ((st = nif_grow(h, h->b_feat, esz * (size_t)h->in_dim * np)) != NIF_OK) return st;
    if ((st = nif_grow(h, h->b_dx, sizeof(float) * (size_t)h->in_dim * n)) != NIF_OK) return st;
    if ((st = nif_grow(h, h->b_out, sizeof(float) * NIF_OUT * n)) != NIF_OK) return st;
    if ((st = nif_grow(h, h->b_feat2, sizeof(float) * NIF_OUT * n)) != NIF_OK) return st;
    if ((st = nif_grow(h, h->b_acts, prec == NIF_FP32 ? sizeof(float) * (size_t)n * h->W * h->H
                                                      : 2 * (size_t)np * kLd * h->H)) != NIF_OK)
        return st;
    if (prec != NIF_FP32 && (st = nif_grow(h, h->b_dys, 2 * (size_t)np * kLd * (h->H + 1))) != NIF_OK) return st;
    if ((st = nif_grow(h, h->b_temp, sizeof(float) * 6 * (size_t)n)) != NIF_OK) return st;
    nif_segment* segs = (nif_segment*)h->b_segs.p;
    nif_linseg* lin = (nif_linseg*)h->b_lin.p;
    nif_label* lab = (nif_label*)h->b_labels.p;
    float* dx = (float*)h->b_dx.p;
    float* out = (float*)h->b_out.p;
    float* dout = (float*)h->b_feat2.p;
    float* dp = (float*)h->b_temp.p;
    if ((st = nif_linearize_run(h, rays, inst_off, n_inst, segs, n_dev, n, lin, s)) != NIF_OK) return st;
    if ((st = nif_labels_run(h, segs, lin, n_dev, n, lab, s)) != NIF_OK) return st;
    if (prec == NIF_FP32) {
        float* feat = (float*)h->b_feat.p;
        float* acts = (float*)h->b_acts.p;
        if ((st = nif_encode_segments_run(h, lin, n_dev, n, feat, NIF_FP32, NIF_FP32, s)) != NIF_OK) return st;
        if ((st = nif_mlp_fwd_fp32_run(h, feat, n_dev, n, out, acts, s)) != NIF_OK) return st;
        if ((st = nif_loss_run(h, out, lab, lin, n_dev, n, dout, s, false)) != NIF_OK) return st;
        if ((st = nif_mlp_bwd_fp32_run(h, feat, n_dev, n, acts, dout, dx, s, false)) != NIF_OK) return st;
    } else {
        uint16_t* acts16 = (uint16_t*)h->b_acts.p;
        if ((st = nif_encode_segments_run(h, lin, n_dev, n, h->b_feat.p, prec, NIF_FP16, s)) != NIF_OK) return st;
        if ((st = nif_mlp_fwd_tc_acts_run(h, h->b_feat.p, prec, n_dev, n, out, acts16, np, kLd, s)) != NIF_OK)
            return st;
        if ((st = nif_loss_run(h, out, lab, lin, n_dev, n, dout, s, false)) != NIF_OK) return st;
        if ((st = nif_mlp_bwd_tc_run(h, dout, acts16, n_dev, n, np, kLd, (uint16_t*)h->b_dys.p, dx, s)) != NIF_OK)
            return st;
    }
    NIF_CK(h, cudaMemsetAsync(dposes, 0, sizeof(float) * 3 * n_inst, s));
    if ((st = nif_encode_segments_dp_run(h, lin, n_dev, n, dx, dp, s)) != NIF_OK) return st;
    if ((st = nif_pose_grad_run(h, segs, lin, dp, n_dev, n, inst_off, n_inst, dposes, s)) != NIF_OK) return st;
    if (prec != NIF_FP32 && (st = nif_unscale_run(h, dposes, 3 * n_inst, s)) != NIF_OK) return st;
    if (loss_host) {
        double acc[16];
        NIF_CK(h, cudaStreamSynchronize(s));
        NIF_CK(h, cudaMemcpy(acc, h->d_lossacc, sizeof(acc), cudaMemcpyDeviceToHost));
        loss_host[0] = acc[8];
        for (int i = 0; i < 5; i++) loss_host[1 + i] = acc[9 + i];
    }
    return NIF_OK;
}

// Fitting the learned deformation field (the paper's future work, Sec. 4;
// the objective is our reading): the segments of the rays under the current
// deformation (poses and field), each segment labelled along its rest segment
// under the target deformation, the task loss of Sec. 2.4 on the network's
// predictions at the current rest segments, and its gradient carried through
// the encoding and the field's inverse into the field (Adam, then the
// Lipschitz projection); with a learning rate for the network, the same
// gradient also trains it (joint).
extern "C" nif_status nif_field_step(nif_handle* h, const nif_pose* poses, int n_inst, const nif_ray* rays,
                                     const int* inst_off, int n_rays, int64_t n_segments,
                                     const nif_pose* target_poses, float lr_field, float lr_grid, float lr_mlp,
                                     double* loss_host, void* stream) {
    if (!h) return NIF_ERR_ARG;
    nif_status st = nif_check_inst(h, poses, n_inst, inst_off, n_rays);
    if (st != NIF_OK) return st;
    if ((st = nif_check_inst(h, target_poses, n_inst, inst_off, n_rays)) != NIF_OK) return st;
    if (h->field_G == 0) return nif_fail(h, NIF_ERR_STATE, "the handle has no field (nif_set_field)");
    if (h->cfg.precision != NIF_FP32 || (h->cfg.flags & NIF_FLAG_MIXED_TRAINING) || h->concat)
        return nif_fail(h, NIF_ERR_STATE, "field fitting runs on FP32 handles of the composed encoding");
    if (n_segments < 1 || !rays || !(lr_field >= 0.f) || !(lr_grid >= 0.f) || !(lr_mlp >= 0.f))
        return nif_fail(h, NIF_ERR_ARG, "n_segments / rays / learning rates");
    const bool joint = lr_grid > 0.f || lr_mlp > 0.f;
    cudaStream_t s = (cudaStream_t)stream;
    if ((st = segment_into_scratch(h, poses, n_inst, rays, inst_off, n_rays, n_segments, false, nullptr, s)) != NIF_OK)
        return st;
    uint32_t* offs = (uint32_t*)h->b_offsets.p;
    const uint32_t* n_dev = offs + n_rays + 1;
    const int64_t n = n_segments;
    if ((st = nif_grow(h, h->b_lin, sizeof(nif_linseg) * n)) != NIF_OK) return st;
    if ((st = nif_grow(h, h->b_lin_t, sizeof(nif_linseg) * n)) != NIF_OK) return st;
    if ((st = nif_grow(h, h->b_labels, sizeof(nif_label) * n)) != NIF_OK) return st;
    if ((st = nif_grow(h, h->b_feat, sizeof(float) * (size_t)h->in_dim * n)) != NIF_OK) return st;
    if ((st = nif_grow(h, h->b_dx, sizeof(float) * (size_t)h->in_dim * n)) != NIF_OK) return st;
    if ((st = nif_grow(h, h->b_out, sizeof(float) * NIF_OUT * n)) != NIF_OK) return st;
    if ((st = nif_grow(h, h->b_feat2, sizeof(float) * NIF_OUT * n)) != NIF_OK) return st;
    if ((st = nif_grow(h, h->b_acts, sizeof(float) * (size_t)n * h->W * h->H)) != NIF_OK) return st;
    if ((st = nif_grow(h, h->b_temp, sizeof(float) * 6 * (size_t)n)) != NIF_OK) return st;
    nif_segment* segs = (nif_segment*)h->b_segs.p;
    nif_linseg* lin = (nif_linseg*)h->b_lin.p;
    nif_linseg* lin_t = (nif_linseg*)h->b_lin_t.p;
    nif_label* lab = (nif_label*)h->b_labels.p;
    float* feat = (float*)h->b_feat.p;
    float* dx = (float*)h->b_dx.p;
    float* out = (float*)h->b_out.p;
    float* dout = (float*)h->b_feat2.p;
    float* acts = (float*)h->b_acts.p;
    float* dp = (float*)h->b_temp.p;
    if ((st = nif_linearize_run(h, rays, inst_off, n_inst, segs, n_dev, n, lin, s)) != NIF_OK) return st;
    if ((st = upload_target_poses(h, target_poses, n_inst, s)) != NIF_OK) return st;
    if ((st = nif_linearize_with_run(h, rays, inst_off, n_inst, h->d_pose_t, FieldView{}, segs, n_dev, n, lin_t, s)) !=
        NIF_OK)
        return st;
    if ((st = nif_labels_run(h, segs, lin_t, n_dev, n, lab, s)) != NIF_OK) return st;
    if ((st = nif_encode_segments_run(h, lin, n_dev, n, feat, NIF_FP32, NIF_FP32, s)) != NIF_OK) return st;
    if ((st = nif_mlp_fwd_fp32_run(h, feat, n_dev, n, out, acts, s)) != NIF_OK) return st;
    if ((st = nif_loss_run(h, out, lab, lin_t, n_dev, n, dout, s, joint)) != NIF_OK) return st;
    if ((st = nif_mlp_bwd_fp32_run(h, feat, n_dev, n, acts, dout, dx, s, joint)) != NIF_OK) return st;
    if (joint && (st = nif_encode_segments_bwd_run(h, lin, n_dev, n, dx, h->d_grad + h->off_tables, s)) != NIF_OK)
        return st;
    if ((st = nif_encode_segments_dp_run(h, lin, n_dev, n, dx, dp, s)) != NIF_OK) return st;
    if ((st = nif_field_grad_run(h, segs, lin, dp, n_dev, n, inst_off, n_inst, h->d_field_g, s)) != NIF_OK) return st;
    if ((st = nif_field_adam_run(h, lr_field, s)) != NIF_OK) return st;
    if (joint && (st = nif_adam_run(h, lr_grid, lr_mlp, s)) != NIF_OK) return st;
    if (loss_host) {
        double acc[16];
        NIF_CK(h, cudaStreamSynchronize(s));
        NIF_CK(h, cudaMemcpy(acc, h->d_lossacc, sizeof(acc), cudaMemcpyDeviceToHost));
        loss_host[0] = acc[8];
        for (int i = 0; i < 5; i++) loss_host[1 + i] = acc[9 + i];
        return latched_status(h);
    }
    return NIF_OK;
}

extern "C" nif_status nif_shadow_rays(nif_handle* h, const nif_ray* rays, const nif_hit* hits, int n,
                                      const float* light_dir_host, float eps, float tmax, nif_ray* shadow_rays,
                                      void* stream) {
    if (!h || n < 0 || (n > 0 && (!rays || !hits || !shadow_rays || !light_dir_host))) return NIF_ERR_ARG;
    const float* L = light_dir_host;
    float len = std::sqrt(L[0] * L[0] + L[1] * L[1] + L[2] * L[2]);
    if (!(len > 0.f) || !(tmax > eps)) return nif_fail(h, NIF_ERR_ARG, "light direction / interval");
    float u[3] = {L[0] / len, L[1] / len, L[2] / len};
    return nif_shadow_rays_run(h, rays, hits, n, u, eps, tmax, shadow_rays, (cudaStream_t)stream);
}

// The sampled batch of one training step of nif_train_step: n_poses poses
// U[-1,1]^3 from step_seed, rays per pose from the sampler, then train_batch.
static nif_status sampled_batch(nif_handle* h, int64_t n_segments, int n_poses, unsigned long long step_seed,
                                nif_pose* poses_out, int* n_rays_out, int* n_hit, cudaStream_t s) {
    std::vector<nif_pose> poses(n_poses);
    for (int i = 0; i < n_poses; i++) {
        uint64_t base = ((0xFFFFull << 32) + (uint64_t)i) * 8ull;
        poses[i].bend = 2.f * host_uniform(step_seed, base) - 1.f;
        poses[i].twist = 2.f * host_uniform(step_seed, base + 1) - 1.f;
        poses[i].taper = 2.f * host_uniform(step_seed, base + 2) - 1.f;
    }
    if (poses_out) std::memcpy(poses_out, poses.data(), sizeof(nif_pose) * n_poses);
    nif_status st;
    // rays per pose: from the segments per ray of a fixed probe (identity pose,
    // a fixed sample stream), so the batch layout depends only on the shape
    if (h->seg_per_ray <= 0.0) {
        const int probe = 8192;
        if ((st = nif_grow(h, h->b_rays, sizeof(nif_ray) * probe)) != NIF_OK) return st;
        if ((st = nif_sample_rays_run(h, 0x5bd1e995ull, 0, probe, (nif_ray*)h->b_rays.p, s)) != NIF_OK) return st;
        int64_t tot = 0;
        const nif_pose identity{0.f, 0.f, 0.f};
        if ((st = segment_into_scratch(h, &identity, 1, (nif_ray*)h->b_rays.p, nullptr, probe, -1, true, &tot, s)) !=
            NIF_OK)
            return st;
        h->seg_per_ray = std::max(0.05, (double)tot / probe);
    }
    int per = (int)std::ceil((double)n_segments / n_poses / h->seg_per_ray * 1.2) + 1;
    int n_rays = per * n_poses;
    if ((st = nif_grow(h, h->b_rays, sizeof(nif_ray) * (size_t)n_rays)) != NIF_OK) return st;
    if ((st = nif_grow(h, h->b_inst, sizeof(int) * (size_t)(n_poses + 1))) != NIF_OK) return st;
    nif_ray* rays = (nif_ray*)h->b_rays.p;
    if ((st = nif_sample_rays_run(h, step_seed, 0, per, rays, s, n_poses)) != NIF_OK) return st;
    k_iota_offsets<<<nif_blocks(n_poses + 1, 256), 256, 0, s>>>((int*)h->b_inst.p, n_poses, per);
    NIF_CK_LAUNCH(h);
    *n_rays_out = n_rays;
    return train_batch(h, poses.data(), n_poses, rays, (const int*)h->b_inst.p, n_rays, n_segments, n_hit, s);
}

extern "C" nif_status nif_train_step(nif_handle* h, int64_t n_segments, int n_poses, unsigned long long step_seed,
                                     float lr_grid, float lr_mlp, nif_pose* poses_out, double* loss_host,
                                     void* stream) {
    if (!h || n_segments < 1 || n_poses < 1) return NIF_ERR_ARG;
    nif_status st;
    if ((h->cfg.flags & NIF_FLAG_MIXED_TRAINING) && (st = check_mixed(h)) != NIF_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    int n_rays = 0;
    if ((st = sampled_batch(h, n_segments, n_poses, step_seed, poses_out, &n_rays, h->d_count, s)) != NIF_OK)
        return st;
    return train_compute(h, n_rays, n_segments, h->d_count, lr_grid, lr_mlp, loss_host, s);
}

// The buffers one training batch lives in, exchanged with the handle's own
// while nif_train_steps builds the next batch beside the current step.
static void swap_batch(nif_handle* h) {
    std::swap(h->b_counts, h->alt_counts);
    std::swap(h->b_offsets, h->alt_offsets);
    std::swap(h->b_temp, h->alt_temp);
    std::swap(h->b_segs, h->alt_segs);
    std::swap(h->b_scan, h->alt_scan);
    std::swap(h->b_rays, h->alt_rays);
    std::swap(h->b_inst, h->alt_inst);
    std::swap(h->b_lin, h->alt_lin);
    std::swap(h->b_labels, h->alt_labels);
    std::swap(h->b_dup, h->alt_dup);
    std::swap(h->b_pts, h->alt_pts);
    std::swap(h->b_sort, h->alt_sort);
    std::swap(h->enc_points, h->alt_enc_points);
}

// The pipeline of nif_train_steps and nif_train_steps_rays: batch i is built
// by build(i, n_hit, stream) into buffer set i % 2 with its hit count in
// counter word 2 + i % 2 (batch 0 on `s`, the others on the third stream
// beside the previous step); step i trains on `s`, then done(i) enqueues on
// `s`. The handle's own buffers are always the set of the next thing enqueued.
// n_rays is read after build(0) has set it; loss_last (nullable) receives the
// last step's loss parts.
template <class Build, class Done>
static nif_status train_pipeline_on(nif_handle* h, int n_steps, const int& n_rays, int64_t n_segments, float lr_grid,
                                    float lr_mlp, double* loss_last, cudaStream_t s, Build build, Done done) {
    nif_status st;
    if ((st = build(0, h->d_count + 2, s)) != NIF_OK) return st;
    NIF_CK(h, cudaEventRecord(h->ev_batch, s));
    // Where the next batch starts, measured: on the FP32 path after the
    // encoding forward (step 3.12 ms; with the step 3.15 ms, where the
    // persistent split-TF32 forward GEMMs lose SMs to it; beside the
    // encoding backward 3.27 ms, where it competes with the backward and the
    // weight gradients, both on whole SMs); the mixed path's forward shares
    // the GPU well and its next batch starts with the step (2.48 ms; 2.55 ms
    // after the encoding forward, 2.91 ms beside the encoding backward).
    const bool early = (h->cfg.flags & NIF_FLAG_MIXED_TRAINING) != 0;
    auto next_batch = [&](int i) -> nif_status {
        swap_batch(h);
        NIF_CK(h, cudaStreamWaitEvent(h->aux2, h->ev_batch, 0));   // batch i built: geometry and cursor free
        NIF_CK(h, cudaStreamWaitEvent(h->aux2, h->ev_step, 0));    // step i - 1 done with this set
        NIF_CK(h, cudaStreamWaitEvent(h->aux2, h->ev_dw[(i + 1) % 2], 0));   // and its late weight gradients
        nif_status r = build(i + 1, h->d_count + 2 + (i + 1) % 2, h->aux2);
        if (r != NIF_OK) return r;
        NIF_CK(h, cudaEventRecord(h->ev_batch, h->aux2));
        return NIF_OK;
    };
    NIF_CK(h, cudaEventRecord(h->ev_step, s));
    for (int i = 0; i < n_steps; i++) {
        const bool more = i + 1 < n_steps;
        if (i > 0) NIF_CK(h, cudaStreamWaitEvent(s, h->ev_batch, 0));      // batch i is built
        if (more && early) {
            if ((st = next_batch(i)) != NIF_OK) return st;
            swap_batch(h);                                                  // back to step i's set
        }
        h->batch_beside = more;                     // the next batch is built beside this step
        st = train_compute(h, n_rays, n_segments, h->d_count + 2 + i % 2, lr_grid, lr_mlp, more ? nullptr : loss_last,
                           s, early ? nullptr : h->ev_step, !more, i % 2);
        h->batch_beside = false;
        if (st != NIF_OK) return st;
        if ((st = done(i, s)) != NIF_OK) return st;
        if (more && !early && (st = next_batch(i)) != NIF_OK) return st;
        if (early) {
            NIF_CK(h, cudaEventRecord(h->ev_step, s));                      // end of step i
            if (more) swap_batch(h);
        }
    }
    return NIF_OK;
}

template <class Build, class Done>
static nif_status train_pipeline(nif_handle* h, int n_steps, const int& n_rays, int64_t n_segments, float lr_grid,
                                 float lr_mlp, double* loss_last, cudaStream_t caller, Build build, Done done) {
    nif_status st;
    // the steps on the high-priority stream (and the weight gradients on its
    // high-priority partner), after the caller's work and before the caller's
    // next; the next batch on the least-priority stream fills what they leave
    const bool prio = h->tune.step_prio != 0;
    const cudaStream_t s = prio ? h->hi : caller;
    const cudaStream_t keep_aux = h->aux;
    if (prio) {
        NIF_CK(h, cudaEventRecord(h->ev_hi_fork, caller));
        NIF_CK(h, cudaStreamWaitEvent(s, h->ev_hi_fork, 0));
        h->aux = h->aux_hi;
    }
    st = train_pipeline_on(h, n_steps, n_rays, n_segments, lr_grid, lr_mlp, loss_last, s, build, done);
    h->aux = keep_aux;
    if (prio) {
        // the join also covers the third stream: its last batch is this call's
        NIF_CK(h, cudaEventRecord(h->ev_hi_join, s));
        NIF_CK(h, cudaStreamWaitEvent(caller, h->ev_hi_join, 0));
    }
    return st;
}

extern "C" nif_status nif_train_steps(nif_handle* h, int n_steps, int64_t n_segments, int n_poses,
                                      unsigned long long first_seed, float lr_grid, float lr_mlp, double* loss_host,
                                      void* stream) {
    if (!h || n_steps < 1 || n_segments < 1 || n_poses < 1) return NIF_ERR_ARG;
    nif_status st;
    if ((h->cfg.flags & NIF_FLAG_MIXED_TRAINING) && (st = check_mixed(h)) != NIF_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    int n_rays = -1;
    auto build = [&](int i, int* n_hit, cudaStream_t bs) -> nif_status {
        int nr = 0;
        nif_status r = sampled_batch(h, n_segments, n_poses, first_seed + (unsigned long long)i, nullptr, &nr, n_hit,
                                     bs);
        if (r != NIF_OK) return r;
        if (n_rays >= 0 && nr != n_rays)
            return nif_fail(h, NIF_ERR_STATE, "training batches of one call differ in ray count");
        n_rays = nr;
        return NIF_OK;
    };
    return train_pipeline(h, n_steps, n_rays, n_segments, lr_grid, lr_mlp, loss_host, s, build,
                          [](int, cudaStream_t) { return NIF_OK; });
}

extern "C" nif_status nif_train_steps_rays(nif_handle* h, int n_steps, const nif_pose* poses, int n_inst,
                                           const nif_ray* rays_host, const int* inst_off, int n_rays,
                                           int64_t n_segments, float lr_grid, float lr_mlp, double* loss_host,
                                           void* stream) {
    if (!h) return NIF_ERR_ARG;
    if (n_steps < 1 || n_rays < 1 || n_segments < 1 || !rays_host)
        return nif_fail(h, NIF_ERR_ARG, "n_steps / n_rays / n_segments / rays");
    nif_status st;
    for (int i = 0; i < n_steps; i++)
        if ((st = nif_check_inst(h, poses ? poses + (size_t)i * n_inst : nullptr, n_inst, inst_off, n_rays)) != NIF_OK)
            return st;
    if ((h->cfg.flags & NIF_FLAG_MIXED_TRAINING) && (st = check_mixed(h)) != NIF_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    // each step's loss parts go to pinned staging on `s` as the step ends
    if (loss_host && h->h_loss_steps < n_steps) {
        if (h->h_loss) cudaFreeHost(h->h_loss);
        h->h_loss = nullptr;
        h->h_loss_steps = 0;
        NIF_CK(h, cudaMallocHost(&h->h_loss, sizeof(double) * 6 * (size_t)n_steps));
        h->h_loss_steps = n_steps;
    }
    auto build = [&](int i, int* n_hit, cudaStream_t bs) -> nif_status {
        nif_status r = nif_grow(h, h->b_rays, sizeof(nif_ray) * (size_t)n_rays);
        if (r != NIF_OK) return r;
        NIF_CK(h, cudaMemcpyAsync(h->b_rays.p, rays_host + (size_t)i * n_rays, sizeof(nif_ray) * (size_t)n_rays,
                                  cudaMemcpyHostToDevice, bs));
        return train_batch(h, poses + (size_t)i * n_inst, n_inst, (const nif_ray*)h->b_rays.p, inst_off, n_rays,
                           n_segments, n_hit, bs);
    };
    auto done = [&](int i, cudaStream_t ds) -> nif_status {
        if (loss_host)
            NIF_CK(h, cudaMemcpyAsync(h->h_loss + 6 * (size_t)i, h->d_lossacc + 8, sizeof(double) * 6,
                                      cudaMemcpyDeviceToHost, ds));
        return NIF_OK;
    };
    if ((st = train_pipeline(h, n_steps, n_rays, n_segments, lr_grid, lr_mlp, nullptr, s, build, done)) != NIF_OK)
        return st;
    if (!loss_host) return NIF_OK;
    NIF_CK(h, cudaStreamSynchronize(s));
    std::memcpy(loss_host, h->h_loss, sizeof(double) * 6 * (size_t)n_steps);
    return latched_status(h);
}

// ---------------------------------------------------------------------------
// Bounds build: each translation unit registers the reader of its device word
// ---------------------------------------------------------------------------
static std::vector<unsigned long long (*)()>& bounds_takers() {
    static std::vector<unsigned long long (*)()> v;
    return v;
}

int nif_bounds_register(unsigned long long (*take)()) {
    bounds_takers().push_back(take);
    return 1;
}

extern "C" nif_status nif_bounds_check(int* enabled, unsigned long long* failures) {
    if (!enabled || !failures) return NIF_ERR_ARG;
    *failures = 0;
#if defined(NIF_BOUNDS) && NIF_BOUNDS
    *enabled = 1;
    if (cudaDeviceSynchronize() != cudaSuccess) {
        cudaGetLastError();
        return NIF_ERR_CUDA;
    }
    for (auto take : bounds_takers()) *failures += take();
#else
    *enabled = 0;
#endif
    return NIF_OK;
}

// ---------------------------------------------------------------------------
// Knobs
// ---------------------------------------------------------------------------
extern "C" nif_status nif_set_knob(nif_handle* h, int knob, double value) {
    if (!h) return NIF_ERR_ARG;
    switch (knob) {
        case NIF_KNOB_WAIT_NS: {
            if (!(value >= 0.0 && value <= 6.0e10)) return nif_fail(h, NIF_ERR_ARG, "wait bound must be in [0, 60 s]");
            const uint64_t ns = (uint64_t)value;
            // after the work already enqueued on any stream of this handle
            NIF_CK(h, cudaDeviceSynchronize());
            NIF_CK(h, cudaMemcpy(h->d_status + 2, &ns, sizeof(ns), cudaMemcpyHostToDevice));
            return NIF_OK;
        }
        case NIF_KNOB_BATCH_AT:
            if (!(value >= 0.0 && value <= 3.0) || value != std::floor(value))
                return nif_fail(h, NIF_ERR_ARG, "batch placement must be 0, 1, 2 or 3");
            h->tune.batch_at = (int)value;
            return NIF_OK;
        case NIF_KNOB_FP32_FUSED:
            if (value != 0.0 && value != 1.0) return nif_fail(h, NIF_ERR_ARG, "fused FP32 forward knob must be 0 or 1");
            h->tune.fp32_fused = h->tune.query_fp32_fused = (int)value;
            return NIF_OK;
        case NIF_KNOB_STEP_BWD_CTAS:
            if (!(value >= -1.0 && value <= 4096.0) || value != std::floor(value))
                return nif_fail(h, NIF_ERR_ARG, "step backward CTA count must be an integer in [-1, 4096]");
            h->tune.step_bwd_ctas = (int)value;
            return NIF_OK;
        case NIF_KNOB_STEP_FWD_CTAS:
            if (!(value >= -1.0 && value <= 4096.0) || value != std::floor(value))
                return nif_fail(h, NIF_ERR_ARG, "step forward CTA count must be an integer in [-1, 4096]");
            h->tune.step_fwd_ctas = (int)value;
            return NIF_OK;
        case NIF_KNOB_DEFER_WEIGHTS:
            if (value != 0.0 && value != 1.0) return nif_fail(h, NIF_ERR_ARG, "deferred weight update knob must be 0 or 1");
            NIF_CK(h, cudaDeviceSynchronize());
            h->tune.defer_wupd = (int)value;
            h->wupd_pending = false;
            return NIF_OK;
        case NIF_KNOB_STEP_PRIORITY:
            if (value != 0.0 && value != 1.0) return nif_fail(h, NIF_ERR_ARG, "step priority knob must be 0 or 1");
            NIF_CK(h, cudaDeviceSynchronize());
            h->tune.step_prio = (int)value;
            return NIF_OK;
        case NIF_KNOB_QUERY_FUSED:
            if (value != 0.0 && value != 1.0) return nif_fail(h, NIF_ERR_ARG, "fused query knob must be 0 or 1");
            h->tune.query_fused = (int)value;
            return NIF_OK;
        case NIF_KNOB_QUERY_SEGS:
            if (!(value > 0.0 && value <= 4096.0)) return nif_fail(h, NIF_ERR_ARG, "segments per ray must be in (0, 4096]");
            h->q_init = value;
            h->q_hint = 0.0;
            h->q_pending = false;
            return NIF_OK;
        case NIF_KNOB_ORDER_BITS:
            if (!(value >= 4.0 && value <= 8.0) || value != std::floor(value))
                return nif_fail(h, NIF_ERR_ARG, "point-order grid bits must be an integer in [4, 8]");
            NIF_CK(h, cudaDeviceSynchronize());
            h->tune.order_bits = (int)value;
            h->enc_points = nif_handle::PointList{};     // a listed order of the old grid is not reused
            h->alt_enc_points = nif_handle::PointList{};
            return NIF_OK;
        case NIF_KNOB_BWD_SPLIT:
            if (value != 0.0 && value != 1.0 && value != 2.0)
                return nif_fail(h, NIF_ERR_ARG, "backward level split must be 0, 1 or 2");
            h->tune.bwd_split = (int)value;
            return NIF_OK;
        case NIF_KNOB_FAIL_ALLOC:
            if (!(value >= 0.0 && value <= 1.0e6) || value != std::floor(value))
                return nif_fail(h, NIF_ERR_ARG, "allocation-failure countdown must be an integer in [0, 1e6]");
            h->fail_alloc = (int)value;
            return NIF_OK;
        case NIF_KNOB_DETERMINISTIC:
            if (value != 0.0 && value != 1.0) return nif_fail(h, NIF_ERR_ARG, "deterministic knob must be 0 or 1");
            if (value == 1.0 && h->concat)
                return nif_fail(h, NIF_ERR_ARG, "deterministic gradients cover the composed reading of Eq. 1 only");
            NIF_CK(h, cudaDeviceSynchronize());
            h->det = value == 1.0;
            h->enc_points = nif_handle::PointList{};     // a listed order is re-made in the mode's own way
            h->alt_enc_points = nif_handle::PointList{};
            return NIF_OK;
        case NIF_KNOB_SEG_SCRATCH:
            if (!(value > 0.0 && value <= 1.0)) return nif_fail(h, NIF_ERR_ARG, "segment scratch scale must be in (0, 1]");
            h->seg_scratch_scale = value;
            return NIF_OK;
        default:
            return nif_fail(h, NIF_ERR_ARG, "unknown knob");
    }
}
