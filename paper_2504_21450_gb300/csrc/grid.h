// grid.h -- host-side state of a vl_grid and the launchers shared between the
// translation units of libvlgt (internal; the public interface is include/vlasov.h).
#pragma once
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <type_traits>
#include <vector>
#include <stdint.h>

#include <algorithm>
#include <string>

#include "common.cuh"
#include "vlasov.h"

namespace vlgt {

// Device buffers of one layout (see common.cuh for what each array holds).
struct Layout {
    uint64_t* ubits = nullptr;   // [nb * RW]
    uint64_t* kbits = nullptr;   // [nb * RW]
    uint32_t* woff = nullptr;    // [nb * RW]
    uint32_t* wcount = nullptr;  // [nb * RW] popcount of ubits per word (scan input)
    uint32_t* cnt = nullptr;     // [nb]
    int64_t* base = nullptr;     // [nb + 1]
    uint8_t* dense = nullptr;    // [nb]
    uint32_t* kcnt = nullptr;    // [nb] kept blocks per id
    void* pool = nullptr;        // [capacity * 64] values in the storage type
    float* scale = nullptr;      // [capacity * 4] power-of-two scale per chunk (16-bit storage)
    uint8_t* keepq = nullptr;    // [capacity * 4] per-chunk keep flags of the last sweep
    int64_t capacity = 0;        // blocks the pool can hold
    int64_t total = 0;           // slots in use (host copy)

    LayoutView view() const { return LayoutView{ubits, kbits, woff, cnt, base, dense, pool, scale}; }
};

struct Grid {
    vl_space_desc space;
    vl_vmesh_desc vmesh;
    double threshold = 0.0;
    vl_storage storage = VL_STORE_F32;
    int codec = 0;      // Codec<codec>: 0 float32, 1 bfloat16, 2 float16
    size_t esize = 4;   // bytes per stored value
    vl_device dev;
    cudaStream_t stream = nullptr;
    GridGeom geom;
    Layout lay[2];   // lay[cur] holds the state, lay[1-cur] the next step's
    int cur = 0;
    bool has_state = false;
    int64_t present = 0;  // blocks present in the current state (host copy)

    // scratch
    StepCounters* counters = nullptr;     // device
    StepCounters* counters_host = nullptr;  // pinned
    uint32_t* tile_flags = nullptr;       // [nb * ntiles]
    uint32_t* tile_pos = nullptr;         // [nb * ntiles]
    uint32_t* item_cnt = nullptr;         // [nb]
    int64_t* item_base = nullptr;         // [nb + 1]
    uint32_t* items = nullptr;            // [nb * ntiles]
    double* item_mass = nullptr;          // [4 * nb * ntiles] (or per CTA of the 3-pass)
    int64_t ntiles_alloc = 0;
    int64_t item_mass_alloc = 0;
    int64_t* host_scalar = nullptr;       // pinned
    int* abort_flag = nullptr;            // device: sticky abort of a captured step sequence
    StepCounters* step_ctr = nullptr;     // device [step_ctr_n]: per-step counters (graphs)
    StepCounters* step_ctr_host = nullptr;  // pinned copy
    int step_ctr_n = 0;
    cudaGraphExec_t graph_exec = nullptr; // cached captured step sequence
    uint64_t graph_key = 0;
    int64_t graph_kernels = 0;            // kernels in the cached graph
    cudaStream_t capture_stream = nullptr;
    cudaStream_t copy_stream = nullptr;   // host-to-device staging of vl_set_blocks
    uint64_t* cta_done = nullptr;         // device [kMaxCtas]: finish time of each fused CTA
    uint64_t* cta_done_host = nullptr;    // pinned copy
    int cta_count = 0;                    // CTAs of the last stamped launch
    int cta_groups = 1;                   // launches stamped back to back (3-pass: three passes)
    float4* ctab = nullptr;               // device [2][3][nvmax] sweep constants
    float4* ctab_host = nullptr;          // pinned staging of the same
    double ctab_dt = -1.0;                // dt the table was built for

    vl_step_stats stats{};
    int64_t launches = 0;                 // kernels launched by the library (running count)
    cudaEvent_t ev_sweep0 = nullptr, ev_sweep1 = nullptr;  // bracket the sweep kernels
    std::vector<cudaEvent_t> graph_ev;  // per captured step: sweep start, sweep end
    std::string last_error;

    void* alloc(size_t bytes);
    void release(void* p);
};

// Running count of kernel launches made by the library (all grids of the process).
void note_launch();
int64_t launch_count();

// Records msg as the grid's last error and returns st.
vl_status fail(Grid* g, vl_status st, const std::string& msg);
vl_status cuda_fail(Grid* g, cudaError_t e, const char* what);

// ---- layout.cu -------------------------------------------------------------
vl_status layout_alloc_meta(Grid* g, Layout& L);
void layout_free(Grid* g, Layout& L);
vl_status layout_ensure_pool(Grid* g, Layout& L, int64_t blocks);
// Frees a layout's value pool and keep flags (its bitmaps stay).
void layout_release_pool(Grid* g, Layout& L);
// Like layout_ensure_pool, but keeps the L.total blocks the pool holds.
vl_status layout_grow_pool(Grid* g, Layout& L, int64_t blocks);
// Counts, offsets and dense flags of L from its ubits (woff, cnt, base, dense);
// returns the total number of slots in *total (synchronises the stream).
vl_status layout_index(Grid* g, Layout& L, int64_t* total);
// next.ubits = 27-cell dilation of cur.kbits (periodic).
void launch_union(Grid* g, const Layout& cur, Layout& next);
// Device-only part of layout_index (no host synchronisation).
void launch_index(Grid* g, Layout& L);
// next.kbits from the per-chunk keep flags; counts kept/dropped blocks and the FP64
// mass of dropped blocks into ctr; sets next.dense bit 1 and next.kcnt; marks ctr done.
void launch_pack_keep(Grid* g, Layout& next, StepCounters* ctr);
// Sets the abort flag and ctr->error bit 3 when L's slot total exceeds capacity.
void launch_capacity_check(Grid* g, const Layout& L, int64_t capacity, StepCounters* ctr);
vl_status set_blocks(Grid* g, int64_t nblocks, const int64_t* off, const uint16_t* ids,
                     const float* vals, int on_device);
vl_status get_block_count(Grid* g, int64_t* n);
// Replaces the blocks of z-planes z0 .. z0+nplanes-1 (wrapping) by the given lists (in
// window order) and keeps every other cell.
vl_status set_blocks_planes(Grid* g, int z0, int nplanes, int64_t nblocks, const int64_t* off,
                            const uint16_t* ids, const float* vals, int on_device);
vl_status get_blocks(Grid* g, int64_t capacity, int64_t* off, uint16_t* ids, float* vals,
                     int on_device);
vl_status get_window(Grid* g, const int* origin, const int* size, int64_t capacity,
                     int64_t* off_out, uint16_t* ids_out, float* vals_out, int on_device,
                     int64_t* count);
vl_status moments(Grid* g, double* out, int on_device);
vl_status tile_features(Grid* g, int edge, float* feat, float* uni);
vl_status total_mass(Grid* g, double* mass);
// Generic scans used by the layout code and the work lists.
void launch_seg_scan(const uint32_t* in, uint32_t* out, uint32_t* seg_total, int64_t seg_len,
                     int64_t nseg, cudaStream_t s, const int* abort);
void launch_base_scan(const uint32_t* seg_total, int64_t* base, int64_t nseg, cudaStream_t s,
                      const int* abort);

// ---- fused.cu / sweep3.cu --------------------------------------------------
struct StepArgs {
    double c_scale[3];  // dt / dx_d
    int order[3];       // physical axis of sweep j
    int limiter;
    int tile[2];
    int ghost = 3;        // GT-k ghost depth (fused form; 3 = exact)
    const float4* walk;   // device [3][nvmax]: WalkConst per axis and velocity index
    const float4* sweep;  // device [3][nvmax]: SweepConst per axis and velocity index
    int nvmax;
    StepCounters* ctr;    // counters of this step
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;  // recorded around the sweep kernels when set
    bool stamp_ctas = false;  // persistent kernels: each CTA records when it ran out of work
    int kernel = 0;       // fused form: 0 plane-batched where it applies and no row-segment
                          // tile is asked for (tile[1]), else row-segment; 1 plane-batched
                          // (VL_EINVAL where it does not apply); 2 row-segment
    bool ev_node = false;  // inside a stream capture: record as event record nodes
};
// Host-side fault injection for tests: true when the environment variable VLGT_FAULT
// lists `what` (comma-separated).  "timeout": the fused kernel reports staging waits
// that are not complete at their first poll as overdue (VL_ETIMEOUT) -- they still
// complete, so no copy is left in flight.
bool fault_requested(const char* what);

// NVTX range over a host scope (phases of a step show up in a timeline profiler; the
// calls cost next to nothing when no tool is attached).
struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange&) = delete;
    NvtxRange& operator=(const NvtxRange&) = delete;
};

// Calls f(std::integral_constant<int, k>{}) for storage codec k (0 float32, 1 bfloat16,
// 2 float16), so that one launch site instantiates the kernel for every codec.
template <class F>
inline void with_codec(int codec, F&& f)
{
    if (codec == 1) f(std::integral_constant<int, 1>{});
    else if (codec == 2) f(std::integral_constant<int, 2>{});
    else f(std::integral_constant<int, 0>{});
}

// Records ev on s; inside a capture as an event record node, which the graph records on
// every replay (a plain record there would only mark a capture dependency).
inline void record_sweep_event(cudaEvent_t ev, cudaStream_t s, bool node)
{
    if (!ev) return;
    if (node) cudaEventRecordWithFlags(ev, s, cudaEventRecordExternal);
    else cudaEventRecord(ev, s);
}
constexpr int kMaxCtas = 4096;  // CTAs of a persistent fused launch, at most
// Tiles of a fused launch: TX (16) cells along axis ax[0], ty along ax[1], ax[2] whole.
struct TileArgs {
    GridGeom G;
    const uint64_t* ubits;
    int ax[3];
    int ntile0, ntile1;
    int ty;
};
void launch_tile_list(Grid* g, const TileArgs& T, int64_t need, int64_t ntiles);
// gt3.cu: the plane-batched GT3 kernel (GT3, streamed axis y or z, no
// velocity block straddling v_d = 0)
bool gt3_applies(const Grid* g, const StepArgs& a);
vl_status run_gt3(Grid* g, const StepArgs& a);
inline bool use_gt3(const Grid* g, const StepArgs& a)
{
    if (a.kernel == 2 || (a.kernel == 0 && a.tile[1] != 0)) return false;  // row-segment tiles asked for
    return gt3_applies(g, a);
}
vl_status fused_worklist_alloc(Grid* g, const StepArgs& a);
// Work-list buffers (g->tile_flags, tile_pos, items) for `need` (block id, tile) pairs.
vl_status worklist_reserve(Grid* g, int64_t need);
// Compacts g->tile_flags ([nb][ntiles]) into g->items / g->item_base (flat: items hold
// b * ntiles + tile).
void launch_items_from_flags(Grid* g, int64_t ntiles, bool flat);
// Work-list buffers of the 3-pass form (its pencil groups; before any captured sequence).
vl_status pass_worklist_alloc(Grid* g);
int tile_rows(const StepArgs& a);
vl_status run_fused(Grid* g, const StepArgs& a);
vl_status run_3pass(Grid* g, const StepArgs& a);
vl_status fused_prepare(Grid* g, const StepArgs& a, int64_t* nwork);
vl_status launch_fused_dense(const GridGeom& G, const LayoutView& in, const LayoutView& out,
                             const int order[3], int limiter, const float4* ctab, int nvmax,
                             const uint32_t* items, const int64_t* item_base, int ntile0,
                             StepCounters* ctr, int device, cudaStream_t stream);
int fused_tile_rows(const int order[3]);
constexpr int kFusedTileX = 16;

}  // namespace vlgt
