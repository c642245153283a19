// mcrt_internal.h -- host-side objects behind the opaque C handles and the
// launchers each .cu file provides.  Not installed; not part of the ABI.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "../../include/mcrt.h"
#include "mcrt_device.cuh"

// One NVTX range per public call (named after it), so a profiler's timeline
// and its kernel filters (ncu --nvtx --nvtx-include "mcrt_trace_camera/")
// see the library's calls; free when no tool is attached.
struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange&) = delete;
    NvtxRange& operator=(const NvtxRange&) = delete;
};

// Host buffers that receive the online-training records of one learned
// trace (mcrt_debug_learned_records); the trace then skips its training.
struct RecordDump {
    int32_t cap = 0;
    float* feat = nullptr;       // cap x 9
    float* dir = nullptr;        // cap x 3
    float* val = nullptr;        // cap x 4: score before, w * omega, own estimate, target
    uint64_t* path = nullptr;    // cap
    int32_t count = 0;           // records the trace produced (may exceed cap)
};

struct mcrt_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    int sm_count = 0;
    size_t l2_bytes = 0;
    uint64_t launches = 0;
    std::string err;
    RecordDump* rec_dump = nullptr;   // set only inside mcrt_debug_learned_records
};

struct mcrt_scene {
    mcrt_ctx* ctx = nullptr;
    int n[3] = {0, 0, 0};
    float h[3] = {0, 0, 0};
    int nb[3] = {0, 0, 0};            // bricks per axis (= level-1 cells)
    float k_clear = 0, ssa_clear = 1, ssa_cloud = 1, g = 0;
    int storage = MCRT_STORAGE_F32;
    void* d_vox = nullptr;            // brick-major field (float or bf16 bits)
    size_t vox_bytes = 0;
    // pyramid: level 1 is filled by the relayout; levels >= 2 by the build
    int levels = 0;                   // built levels (0 = none)
    float* d_pyr = nullptr;           // all levels, concatenated; the minorant levels follow at + pyr_capacity
    size_t pyr_capacity = 0;          // floats allocated
    std::vector<size_t> lev_off;      // offset of level L (index L), floats
    std::vector<int> lev_dims;        // 3 ints per level (index 3L)
    // the paper's octree (built on request): 2^L voxels per cell and axis
    int oct_levels = 0;               // built levels (0 = none)
    float* d_oct = nullptr;           // max levels, then the min levels at + oct_capacity
    size_t oct_capacity = 0;
    std::vector<size_t> oct_off;      // offset of level L (index L), floats
    std::vector<int> oct_dims;        // 3 ints per level (index 3L)
    uint2* d_oleaf = nullptr;         // leaf map over the octree's level-1 cells
    // leaf map for one (tau~, finest level, grid); d_leaf serves the
    // pyramid, d_oleaf the octree
    uint2* d_leaf = nullptr;
    bool leaf_valid = false;
    float leaf_tau = 0;
    int leaf_finest = -1;
    int leaf_grid = MCRT_GRID_PYRAMID;
    // bumped whenever something a device scene record holds changes (leaf
    // map rebuilt, octree or pyramid rebuilt, ground or phase changed), so
    // that saved records (batch plans) know to refresh
    uint64_t gen = 0;
    float albedo = 0;
    int clear_phase = 0;              // MCRT_PHASE_HG or MCRT_PHASE_RAYLEIGH
    float sun_zenith = 0, sun_azimuth = 0;
    float sun[3] = {0, 0, 1};
    // heightfield ground (null: flat)
    float* d_hf = nullptr;
    float* d_hpyr = nullptr;
    int hn[2] = {0, 0};
    float hmax = 0;
    int hlev = 0;
    int hoff[mcrt::kMaxHfLevels] = {};
};

struct mcrt_tally {
    mcrt_ctx* ctx = nullptr;
    int ncells = 0, nq = 0;
    uint64_t n_per_cell = 0;
    double* d_s1 = nullptr;
    double* d_s2 = nullptr;
    unsigned long long* d_counters = nullptr;   // 16 counters
    void* d_work = nullptr;                      // WorkState
    double* d_out = nullptr;                     // finalize scratch (mean, se)
    float kernel_ms = 0;
    std::vector<uint64_t> cell_n;                // per-cell path counts (batches) ...
    unsigned long long* d_cell_n = nullptr;      // ... and their device copy
};

struct mcrt_proposal {
    mcrt_ctx* ctx = nullptr;
    float* d_params = nullptr;     // FP32 master parameters (11,560)
    float* d_m = nullptr;          // Adam first moments
    float* d_v = nullptr;          // Adam second moments
    float* d_grad = nullptr;       // gradient accumulator
    float* d_loss = nullptr;       // loss accumulator (1 float)
    void* d_wbf = nullptr;         // padded BF16 inference weights
    float* d_bias = nullptr;       // padded FP32 biases
    int step = 0;                  // Adam steps taken
    int train_mode = MCRT_TRAIN_TENSOR;   // gradient kernel: tensor cores (BF16) or FP32
};

namespace mcrt {

constexpr int kNumCounters = 32;
constexpr int kMlpParams = 11560;

// Work distribution and status shared by all blocks of a trace launch.
struct WorkState {
    unsigned long long next;   // next path id to claim
    int status;                // 0 ok, 1 deadline, 2 cancelled
    int pad;
};

// One item of a batch: a scene (with its band's gas absorption and sun), a
// chunk-aligned range of work ids, and its own Philox key; path i of the
// item draws the numbers path i of a single trace with that seed would.
struct BatchItem {
    DevScene S;
    unsigned long long begin;   // first work id (chunk aligned)
    unsigned long long npaths;
    uint2 key;
};

// Launch parameters of the tracer.
struct TraceParams {
    DevScene S;
    unsigned long long total;  // paths
    uint32_t chunk;            // paths per claim
    uint2 key;                 // Philox key (seed)
    int max_order;
    int sun_mode;
    uint32_t max_steps;
    int rare_batch;            // lanes waiting for a rare phase that trigger it
    int min_steppers;          // below this many stepping lanes, run rare phases anyway
    // camera
    int width, height;
    uint32_t spp;
    float cam_pos[3], cam_f[3], cam_r[3], cam_u[3];
    float tan_half, aspect;    // tan(fov/2), height/width
    float inv_width, inv_height;
    float Lz;
    // learned proposal (wavefront rounds): paths stop at their first
    // n_learned volume vertices, the network evaluates the queue, and the next
    // launch resumes them
    int learned;               // 0 plain HG; 1 learned rounds
    int resume;                // 0: fresh paths [0, total); 1: queue slots [0, total)
    int n_learned;             // volume vertices per path drawn with the network
    float mis_alpha;           // HG share of the one-sample MIS mixture
    unsigned long long path_base;  // first path id of the batch (record / final-score index origin)
    const uint4* qin;          // resumed states, 4 x uint4 per slot
    const uint4* qin_feat;     // their feature rows (16 bf16 = 2 uint4)
    const float* qin_mix;      // their mixture parameters (48 floats: mu, kappa, weight CDF, pi C(kappa) per lobe)
    uint4* qout;               // suspended states
    uint4* qout_feat;          // suspended feature rows
    unsigned* qout_count;
    unsigned qout_cap;
    // training records (written when a resumed vertex samples its direction)
    uint4* rec_feat;           // feature rows
    float* rec_dir;            // 3 floats
    float* rec_val;            // 4 floats: score before the vertex, w*omega, own estimate, path index
    unsigned* rec_count;
    unsigned rec_cap;
    unsigned rec_slots;        // only queue slots below this are recorded
    float* final_score;        // per path of the batch
    const float* pyr1;         // level-1 majorants (features)
    const float* pyr2;         // level-2 (or top) majorants
    int d1[3], d2[3];
    int lev2;                  // level of pyr2
    // batches (flux sensor): items sorted by begin
    const BatchItem* items;
    int n_items;
    // camera: pixel of each claim rank (null: raster order)
    const uint32_t* pix_order;
    // outputs
    double* s1;
    double* s2;
    unsigned long long* counters;
    WorkState* work;
    // control
    unsigned long long deadline_ns;       // 0 = none
    const volatile int* cancel;
};

// Rare phases (path start, ray start, vertex) of a warp run once this many
// of its lanes wait for them (the default when a caller passes 0), or when
// fewer than 33 - that many lanes are stepping.  Launch shape only.
constexpr int kDefaultRareBatch = 10;
inline void set_rare_batch(TraceParams& P, int requested)
{
    P.rare_batch = requested > 0 ? requested : kDefaultRareBatch;
    P.min_steppers = 33 - P.rare_batch;
}

enum Sensor { kCamera = 0, kFlux = 1 };

// Launchers (return cudaError of the launch).
cudaError_t launch_relayout(const float* src, const mcrt_scene* sc, cudaStream_t st);
cudaError_t launch_reduce_level(const float* prev, const int* prev_dims, float* out, const int* dims, bool min_level,
                                cudaStream_t st);
cudaError_t launch_leafmap(const mcrt_scene* sc, float tau, int finest, int grid, cudaStream_t st);
cudaError_t launch_octree(const mcrt_scene* sc, const DevScene& S, cudaStream_t st);
cudaError_t launch_hf_pyramid(const float* h, int nx, int ny, float* pyr, const int* off, int levels, cudaStream_t st);
cudaError_t launch_hf_check(const float* h, long long n, float top, int* bad, cudaStream_t st);
cudaError_t launch_debug_terrain(const DevScene& S, const float* o, const float* d, int n, float* t, cudaStream_t st);
cudaError_t launch_debug_terrain_height(const DevScene& S, const float* xy, int n, float* zn, cudaStream_t st);
cudaError_t launch_trace(const TraceParams& P, int sensor, bool bf16, bool count, int grid, int block,
                         cudaStream_t st);
int trace_blocks_per_sm(int sensor, bool bf16, bool count, bool terrain, bool extra, int block);
cudaError_t launch_trace_learned(const TraceParams& P, int sensor, bool bf16, int grid, int block, cudaStream_t st);
int trace_learned_blocks_per_sm(int sensor, bool bf16, int block);
cudaError_t launch_targets(const float* rec_val, const float* final_score, unsigned n, float* tgt, cudaStream_t st);
cudaError_t launch_trace_batch(const TraceParams& P, bool bf16, bool count, bool dalpha, int grid, int block,
                               cudaStream_t st);
int trace_batch_blocks_per_sm(bool bf16, bool count, bool dalpha, int block);
cudaError_t launch_finalize(const double* s1, const double* s2, double n, int count, const unsigned long long* cell_n,
                            int nq, double* out, cudaStream_t st);
// Default paths per claim (mcrt_trace_opts.chunk = 0).  A lane traces the
// paths of its chunk one after another, so with few paths per resident
// lane long chunks stretch the launch's tail (a chunk of one cloudy pixel
// holds several long random walks); with many, short chunks cost claims.
// Thresholds from GB300 measurements on the cumulus field: chunk 1 below
// 48 paths per lane, 2 below 160, 4 below 400, else 8 (the most the FP32
// chunk sums are bounded for); camera chunks divide spp.
inline uint32_t auto_chunk(unsigned long long total, unsigned long long lanes, uint32_t spp)
{
    const double per_lane = lanes ? (double)total / (double)lanes : 0.0;
    uint32_t c = per_lane < 48.0 ? 1u : (per_lane < 160.0 ? 2u : (per_lane < 400.0 ? 4u : 8u));
    if (spp) {
        if (c > spp) c = spp;
        while (spp % c) --c;
    }
    return c;
}

bool bounds_checked_build();
cudaError_t read_bounds_violations(unsigned* count, unsigned* first_code);
int order_tiles(int width, int height, int* tiles_x);
cudaError_t launch_view_cost(const TraceParams& P, bool bf16, float* cost, cudaStream_t st);
cudaError_t launch_expand_order(const uint32_t* tiles, const uint32_t* prefix, int n, int width, int height,
                                uint32_t* order, cudaStream_t st);
cudaError_t launch_shard_order(const uint32_t* order, uint32_t n_out, uint32_t stride, uint32_t offset,
                               uint32_t* out, cudaStream_t st);
cudaError_t launch_debug_dda(const DevScene& S, const float* o, const float* d, int cap, int* cells,
                             float* tio, int* count_status, bool bf16, cudaStream_t st);
cudaError_t launch_debug_philox(const uint32_t* ctr, const uint32_t* key, uint32_t* out, size_t n,
                                cudaStream_t st);

DevScene make_dev_scene(const mcrt_scene* sc, float k_gas);

// Camera trace scheduled as a wavefront (wavefront.cu): `slots` queue
// entries per stage, rounds of flight, vertex and start kernels until every
// path has ended.  ms: device time from the first to the last kernel.
struct WavefrontStats {
    float ms;
    unsigned rounds;
    unsigned overflow;             // 1: a queue was full; 2: too many rounds
    unsigned long long launches;
};
cudaError_t wavefront_camera(const TraceParams& P, bool bf16, unsigned slots, int sm_count, cudaStream_t st,
                             WavefrontStats* stats);
int wavefront_blocks_per_sm(bool bf16);

// Option checks shared by the trace entry points (status and message as
// mcrt_trace_camera reports them), and the leaf map of (tau~, finest level,
// grid), rebuilt in place when another one is current.
int check_opts(mcrt_scene* sc, const mcrt_trace_opts* o, const char* who);
int ensure_leaf(mcrt_scene* sc, float tau, int finest, int grid);

// learned proposal network
size_t mlp_packed_bf16_elems();
size_t mlp_packed_bias_elems();
// mix: 40 floats per row (mu, kappa, pi per lobe), or with tracer_layout
// 48 (mu, kappa, weight CDF, pi C(kappa)) as the learned trace reads them.
cudaError_t launch_mlp_infer(const void* wpacked, const float* bpacked, const void* feat, int n, float* mix,
                             float* raw, int sm_count, cudaStream_t st, bool tracer_layout = false);
cudaError_t launch_mlp_train_tc(const void* wpacked, const float* bpacked, const float* params, const void* feat,
                                const float* dirs, const float* tgt, int n, float scale, float* grad, float* loss,
                                int sm_count, cudaStream_t st);
// 1 in *err if an MMA wait of the tensor-core network kernels ran out since
// the last call (then cleared); synchronises the stream.
cudaError_t tc5_take_error(int* err, cudaStream_t st);
cudaError_t launch_mlp_train(const float* params, const void* feat, const float* dirs, const float* tgt, int n,
                             float scale, float* grad, float* loss, int sm_count, cudaStream_t st);
cudaError_t launch_adam(float* p, float* m, float* v, const float* g, int n, float lr, float b1, float b2, float eps,
                        int t, cudaStream_t st);
cudaError_t launch_pack(const float* p, void* w, float* b, cudaStream_t st);
cudaError_t launch_xavier(float* p, uint64_t seed, cudaStream_t st);
cudaError_t launch_f32_to_bf16_rows(const float* src, int n, int cols, void* dst, int ld, cudaStream_t st);

}  // namespace mcrt
