/*
 * vlasov.h -- C ABI of libvlgt, a single-GPU (GB300, sm_103a) implementation of the
 * spatial translation step of a 6D Vlasov solver in its coalesced-ghost form.
 *
 * What the library computes (arXiv:2504.21450, "Coalescing MPI communication in 6D
 * Vlasov simulations: solving ghost domains in Vlasiator"):
 *   - Section 2 / Eq. 1: the v . grad_x f term of the Vlasov equation, advanced by three
 *     Cartesian shears per time step (Section 2.1), each a mass-conserving
 *     semi-Lagrangian remap with a piecewise-parabolic fit on a stencil of 2 cells that
 *     writes into the cell itself and its downwind face neighbour; dt is limited so that
 *     one face neighbour suffices (|v_d| dt / dx_d <= 1).
 *   - Section 2: a sparse velocity space of 4x4x4 (64-value) blocks per spatial cell,
 *     added where a neighbour can send content and removed below a sparsity threshold.
 *   - Section 3: Ghost Translation -- each spatial tile loads its ghost halo once, wide
 *     enough for all three sweeps, and computes on the ghost cells (the "fused" form),
 *     instead of exchanging ghosts between sweeps (the classical, "3-pass" form).
 *
 * Conventions
 *   - Spatial cell index c = x + nx*(y + ny*z); the grid is periodic in all dimensions.
 *   - Block id b = bx + nbx*(by + nby*bz) with nbx = nv[0]/4 etc. (at most 65536 ids).
 *   - The 64 values of a block are ordered vx fastest, then vy, then vz.  Velocity cell
 *     centres: v_d = vmin[d] + (i_d + 1/2) dv[d].
 *   - Transfer format ("per-cell lists"): cell_offsets[ncells+1] (int64, prefix sums),
 *     block_ids[nblocks] (uint16, strictly increasing within a cell), values[nblocks*64]
 *     (float32).  The library stores f in its own layout and converts on set/get.
 *   - Every call returns a vl_status; no call aborts, traps or exits.  After an error
 *     vl_last_error() describes it.  A grid is used by one host thread at a time.
 *   - Work is queued on the grid's stream; calls that return data to the host
 *     synchronise that stream.  Device pointers must be valid on the grid's device.
 *   - Memory: the library owns the device memory of a grid and obtains it through the
 *     caller's allocator callbacks (or cudaMalloc when they are NULL); the caller owns
 *     every buffer it passes in.
 */
#ifndef VLASOV_H
#define VLASOV_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct vl_grid vl_grid; /* opaque, owned by the library */

typedef enum {
    VL_OK = 0,
    VL_EINVAL = 1,     /* bad argument (null pointer, bad size, unsorted ids, ...) */
    VL_ENOMEM = 2,     /* the allocator returned NULL */
    VL_ECFL = 3,       /* max |v_d| dt / dx_d > 1 (Section 2.1's one-neighbour limit) */
    VL_ECAPACITY = 4,  /* a pre-sized buffer was too small (recoverable) */
    VL_ETIMEOUT = 5,   /* a bounded device wait ran out */
    VL_ECUDA = 6,      /* a CUDA runtime call failed */
    VL_ESTATE = 7      /* call not valid in the grid's current state */
} vl_status;

/* Storage of f in device memory (the paper fixes none; the arithmetic of a sweep is
 * float32 in every form).  The 16-bit forms keep q = f / s rounded to nearest even,
 * with one power-of-two float32 scale s per chunk -- the 16 values of one vz plane of a
 * 4x4x4 block in one cell: whoever writes a chunk sets s to the smallest power of two
 * >= its largest |f| (at least 2^-126, at most 2^127, 1 for an all-zero chunk), so
 * every code lies in [-1, 1].  Every value read through this interface is float32
 * (q * s); every value written is rounded to the storage type.  The fused form rounds
 * once per step, the 3-pass form after each of its three sweeps.  The scales take 4
 * bytes per 32 bytes of codes. */
typedef enum {
    VL_STORE_F32 = 0,          /* f stored as float32 */
    VL_STORE_BF16_SCALED = 1,  /* bfloat16 code x power-of-two float32 scale per chunk */
    VL_STORE_F16_SCALED = 2    /* float16 code x power-of-two float32 scale per chunk */
} vl_storage;

typedef enum {
    VL_FORM_FUSED = 0,  /* Ghost Translation: one tile+halo load, x->y->z in one kernel */
    VL_FORM_3PASS = 1,  /* classical: one HBM round trip per sweep direction */
    VL_FORM_AUTO = 2    /* pick per workload: the first steps run for a workload probe
                           each candidate -- fused with the plane-batched kernel (where it
                           applies), fused row-segment kernel with 16-row tiles (orders
                           ending in z) and with 8-row tiles, 3-pass (FP32 storage only) --
                           with one warm-up and one timed step each, over as many calls as
                           it takes (every probe step advances the real state; the
                           candidates compute the same result).  With FP32 storage a prior
                           from Section 3.3's ghost-work count rules out, unprobed, a fused
                           candidate whose tile sweeps more than 3 times as many cells per
                           useful update as the 3-pass form (it moves a third of the bytes,
                           so it cannot win); a single remaining candidate is taken
                           without probing.  Candidates are compared by the time of their
                           sweep kernels per updated cell in the timed step (the other
                           phases are the same for all of them, and a step that grows a
                           pool spends host time that says nothing about the form); the
                           fastest is cached per workload
                           key (grid, velocity mesh, order, limiter, storage, slots per
                           cell rounded to a power of two); with the environment variable
                           VLGT_TUNE_CACHE naming a file the choices also persist across
                           processes (JSON lines).  Exact forms only: it requires
                           ghost = 3 */
} vl_form;

/* Spatial box: n cells per dimension, cell size dx, origin x0 (periodic). */
typedef struct {
    int n[3];
    double dx[3];
    double x0[3];
} vl_space_desc;

/* Velocity mesh: nv cells per dimension (multiples of block[d]), lower corner vmin,
 * cell size dv; block must be {4,4,4} (Section 2's 64-element blocks). */
typedef struct {
    int nv[3];
    double vmin[3];
    double dv[3];
    int block[3];
} vl_vmesh_desc;

/* Device memory and stream.  alloc/free may be NULL (then cudaMalloc/cudaFree are
 * used).  alloc must return memory aligned to at least 256 bytes.  stream is a
 * cudaStream_t (NULL: the legacy default stream); device is the CUDA device ordinal. */
typedef struct {
    void* (*alloc)(size_t bytes, void* ctx);
    void (*free)(void* ptr, void* ctx);
    void* ctx;
    void* stream;
    int device;
} vl_device;

/* Options of vl_translate; a NULL pointer means all defaults (the zero-initialised
 * struct is NOT the default: use vl_translate_opts_default). */
typedef struct {
    int form;       /* vl_form; default VL_FORM_FUSED */
    int limiter;    /* 1 (default): monotonicity limiter on; 0: linear PPM (dense
                       velocity meshes only: without the limiter content can reach
                       cells outside the 27-cell block union) */
    int ghost;      /* ghost depth k of GT-k (Section 3.2), default 3.  3 (GT3) is exact:
                       the step equals the classical sweep-by-sweep one.  1 and 2 (GT1,
                       GT2) exist in the fused form with FP32 storage (else VL_EINVAL):
                       the first sweep runs only on the tile's rows and the k rows
                       beyond it on each side along the second sweep axis; rows further
                       out enter the second sweep's stencils with their pre-step values,
                       so the result is approximate and its error depends on the tile
                       shape (16 x `tile[1]` cells along the first two sweep axes, the
                       third axis whole) */
    int tile[2];    /* fused tile extent along the first two sweep axes; 0 = default */
    int check;      /* 1: synchronise after the call and report device-side errors */
    int graph;      /* 1: run the nsteps steps as one captured CUDA graph with no host
                       synchronisation between steps.  The pools are sized to at least
                       `capacity` blocks beforehand (they never shrink); a step that
                       would need more slots than they hold is detected on the device,
                       the state stays at the last complete step, the pools grow and
                       the remaining steps run again.  The graph is cached and replayed
                       by later calls with the same step count, form, order and pools. */
    int kernel;     /* fused form, which kernel: 0 (default) the plane-batched kernel (16 x 16
                       tiles) where it applies -- GT3, streamed axis y or z, no
                       velocity block straddling v_d = 0, tile[1] = 0 -- else the row-segment
                       kernel; 1 the plane-batched kernel (VL_EINVAL where it does not
                       apply); 2 the row-segment kernel (tile rows from tile[1]) */
    int64_t capacity; /* graph mode: blocks per layout; 0 = 1.25 x the current slots */
    int reserved[4];
} vl_translate_opts;

/* Counters of the last vl_translate call (FP64 sums on the device). */
typedef struct {
    int64_t steps;          /* steps done by the last call */
    int64_t blocks;         /* blocks present after the last step */
    int64_t union_blocks;   /* blocks of the last step's 27-cell union (before pruning) */
    int64_t dropped_blocks; /* blocks removed by the sparsity rule in the last step */
    double mass;            /* total mass after the last step (kept blocks) */
    double dropped_mass;    /* mass removed by the sparsity rule over the whole call */
    double mass_before;     /* total mass before the first step of the call */
    double device_ms;       /* device time of the call's steps (CUDA events) */
    double sweep_ms;        /* device time of the sweep kernels alone (the hot loop) */
    double index_ms;        /* block union, slot indexing and work lists */
    double prune_ms;        /* sparsity rule and dropped-mass accounting */
    int64_t launches;       /* kernels the library launched during the call */
    int64_t graph_replays;  /* graph mode: captured sequences launched (incl. re-runs) */
    int64_t capacity_regrows; /* graph mode: capacity overflows recovered from */
    int64_t capacity;       /* graph mode: blocks per layout at the end of the call */
    int form_used;          /* vl_form of the last step (after autotuning) */
    int tile_rows_used;     /* fused form: tile rows along the second sweep axis */
    double tune_ms[4];      /* autotuner probes (sweep kernels' ms in the timed probe
                               step): fused plane-batched kernel,
                               fused row-segment kernel with 16-row and 8-row tiles,
                               3-pass; 0 = not applicable, -1 = ruled out by the
                               ghost-work prior (VL_FORM_AUTO) */
    int64_t updates;        /* phase-space cell updates of the call: velocity cells present
                               at the start of each step, summed over its steps */
    double tail_ms;         /* steps run one by one: summed over steps, the time from the
                               first to the last CTA of a persistent sweep kernel running
                               out of work (the single-GPU counterpart of the paper's wait
                               time, Table 1) -- the fused kernel, or the three passes of
                               the 3-pass form on a sparse state (work-list mode); 0
                               otherwise */
    int kernel_used;        /* fused form: 1 plane-batched kernel, 2 row-segment kernel */
    int reserved_stats;
} vl_step_stats;

void vl_translate_opts_default(vl_translate_opts* opts);

/* Create an empty grid (no blocks).  sparsity_threshold is absolute: after each step
 * a block is kept iff its largest value is >= the threshold (Section 2); 0 keeps every
 * block that the union created.  storage selects float32 or a scaled 16-bit form (see
 * vl_storage); with a 16-bit form the threshold is compared with the stored values.
 * Errors: VL_EINVAL (bad descriptor, block != {4,4,4}, storage), VL_ECUDA, VL_ENOMEM. */
vl_status vl_grid_create(const vl_space_desc* space, const vl_vmesh_desc* vmesh,
                         double sparsity_threshold, vl_storage storage,
                         const vl_device* device, vl_grid** out);

/* Free the grid and all device memory it holds.  NULL is accepted. */
vl_status vl_grid_destroy(vl_grid* grid);

/* Replace the grid's state by the given per-cell lists.  on_device = 0: host pointers
 * (copied synchronously; when `values` is page-locked host memory -- cudaHostAlloc,
 * cudaMallocHost, cudaHostRegister -- the scatter kernel reads it in place, over
 * NVLink-C2C on a Grace host, else it is staged through device buffers); 1: device
 * pointers on the grid's device (read on its stream before the call returns).
 * nblocks = cell_offsets[ncells].  values are float32; with
 * 16-bit storage each chunk of 16 is rounded to it with the scale of its own largest
 * magnitude.
 * Errors: VL_EINVAL (offsets not non-decreasing, ids out of range or not strictly
 * increasing within a cell), VL_ENOMEM, VL_ECUDA. */
vl_status vl_set_blocks(vl_grid* grid, int64_t nblocks, const int64_t* cell_offsets,
                        const uint16_t* block_ids, const float* values, int on_device);

/* Number of blocks currently present (synchronises the grid's stream). */
vl_status vl_get_block_count(vl_grid* grid, int64_t* nblocks);

/* Copy the state out as per-cell lists into caller-allocated buffers of at least
 * `capacity` blocks (cell_offsets: ncells+1 entries).  on_device as in vl_set_blocks
 * (page-locked host `values` are written in place by the gather kernel).
 * Errors: VL_ECAPACITY when capacity < vl_get_block_count. */
vl_status vl_get_blocks(vl_grid* grid, int64_t capacity, int64_t* cell_offsets,
                        uint16_t* block_ids, float* values, int on_device);

/* Replace the blocks of the z-planes z0 .. z0+nplanes-1 (wrapping periodically) by the
 * given per-cell lists and keep every other cell: the ghost update of a decomposition of
 * the spatial domain into z-slabs (Section 3: one coalesced ghost update per step, from
 * the neighbours' boundary planes, which vl_get_blocks_window reads).  The lists cover
 * nx*ny*nplanes cells in window order (x fastest, then y, then the planes in order),
 * nblocks = cell_offsets[nx*ny*nplanes]; on_device as in vl_set_blocks.  When the
 * lists hold exactly the blocks the window already holds, their values are written into
 * the existing slots (work of the order of the window); otherwise the layout is rebuilt
 * from the whole state's lists on the device (work and scratch memory of the order of
 * the state; 16-bit codes of the other cells come back unchanged, since re-deriving a
 * chunk's scale from its decoded values reproduces its codes).  Errors: VL_ESTATE (no state), VL_EINVAL, VL_ENOMEM, VL_ECUDA. */
vl_status vl_set_blocks_planes(vl_grid* grid, int z0, int nplanes, int64_t nblocks,
                               const int64_t* cell_offsets, const uint16_t* block_ids,
                               const float* values, int on_device);

/* Per-cell lists of a box window: the cells origin[d] + [0, size[d]) (wrapping
 * periodically), x fastest, 1 <= size[d] <= n[d].  Same formats, ownership and errors as
 * vl_get_blocks; cell_offsets has size[0]*size[1]*size[2]+1 entries.  Used to sample a
 * large state (checkpointing a sub-domain, comparing a window with a reference). */
vl_status vl_get_block_count_window(vl_grid* grid, const int origin[3], const int size[3],
                                    int64_t* nblocks);
vl_status vl_get_blocks_window(vl_grid* grid, const int origin[3], const int size[3],
                               int64_t capacity, int64_t* cell_offsets, uint16_t* block_ids,
                               float* values, int on_device);

/* Advance the state by nsteps translation steps of length dt with the sweeps in the
 * given order (a permutation of "xyz"; Section 2.1 uses z->x->y).  Each step: 27-cell
 * block union, the three PPM shears (fused GT3 tile kernel or three passes), then the
 * sparsity rule with FP64 accounting of the dropped mass.
 * Errors: VL_ECFL (Section 2.1's one-neighbour limit), VL_EINVAL, VL_ENOMEM, VL_ECUDA. */
vl_status vl_translate(vl_grid* grid, double dt, const char* order, int nsteps,
                       const vl_translate_opts* opts);

/* Checkpoint (the paper restarts its runs from a saved state, Section 4.2): the grid's
 * state as one self-describing host buffer -- a header (magic "VLGT", format version 3,
 * spatial extents, velocity mesh, cell and velocity sizes, threshold, block count,
 * storage type, block ids) followed by the per-cell lists (cell_offsets, values,
 * block_ids) of vl_get_blocks.  A restarted run continues bit for bit: with 16-bit
 * storage the decoded values determine the codes and scales (a chunk's scale re-derived
 * from its decoded values reproduces its codes exactly).
 * vl_export with buf == NULL stores the required size in *size; otherwise *size must
 * hold the buffer's size (VL_ECAPACITY when too small) and receives the bytes written.
 * vl_import replaces the state of a grid with the same extents, velocity mesh and
 * storage type (VL_EINVAL otherwise, or for a damaged buffer). */
vl_status vl_export(vl_grid* grid, void* buf, size_t* size);
vl_status vl_import(vl_grid* grid, const void* buf, size_t size);

/* Velocity moments per cell (particle mass 1), FP64: out[c*7 + k] for
 * k = n, nVx, nVy, nVz, Pxx, Pyy, Pzz with n = sum f dv^3, nV_d = sum v_d f dv^3,
 * P_dd = sum (v_d - V_d)^2 f dv^3.  on_device as in vl_set_blocks. */
vl_status vl_moments(vl_grid* grid, double* out, int on_device);

/* FP64 total mass (sum f dx^3 dv^3) of the current state (synchronises). */
vl_status vl_mass(vl_grid* grid, double* mass);

/* Counters of the last vl_translate (synchronises). */
vl_status vl_stats(vl_grid* grid, vl_step_stats* stats);

/* One translation step that allocates no device memory.
 *
 * The paper has no counterpart to this call: it exists for callers that cannot allocate,
 * such as a runtime that owns the whole device memory budget, an embedding host whose
 * allocator this library cannot reach, or code that must not touch the device heap
 * between two steps.
 *
 * It runs the fused Ghost Translation kernel (the three PPM sweeps, Section 3) once on a
 * DENSE velocity space (every cell holds every block id), without the sparsity rule.
 * f_in and f_out are device pointers owned by the caller, each
 * (nv[0]/4)*(nv[1]/4)*(nv[2]/4) * ncells * 64 floats, in the library's storage order:
 * f[((b*4 + q)*ncells + c)*16 + l] for block id b, vz index q within the block, cell c
 * and in-plane index l = vx + 4*vy within the block.  They must not overlap.  *mass_out
 * (device pointer) receives the FP64 total mass of f_out (sum of values times
 * dx^3 dv^3).  Work is queued on `stream` (a cudaStream_t, NULL = legacy default stream)
 * of the current device; the call does not synchronise.
 *
 * Everything else the kernel needs (work list, layout tables, sweep constants, counters)
 * lives in one static device array of VL_NOALLOC_SCRATCH_BYTES, which every GPU that
 * loads the library holds until the process exits.  The first call on a device looks
 * up that array's device address (setup); make that first call before any stream
 * capture.  All calls share the array and each one overwrites it, so calls whose work
 * overlaps on the GPU (on different streams, or from different host threads) race: order
 * them on one stream.
 * Errors: VL_EINVAL (null pointer, bad descriptor or order, f_in == f_out), VL_ECFL,
 * VL_ECAPACITY (the work list of this grid does not fit in the static array: at most
 * about 1 MiB for nb*(21 + 4*tiles) bytes, with tiles = ceil(n_a/16)*ceil(n_b/TY) over
 * the first two sweep axes, TY = 16 when the order ends in z, else 8), VL_ECUDA. */
#define VL_NOALLOC_SCRATCH_BYTES (1u << 20)
vl_status vl_translate_dense_noalloc(const vl_space_desc* space, const vl_vmesh_desc* vmesh,
                                     double dt, const char* order, int limiter,
                                     const float* f_in, float* f_out, double* mass_out,
                                     void* stream);

/* ---- learned cost model --------------------------------------------------------------
 * The paper weighs each spatial cell by the complexity of its velocity space when it
 * balances load (Section 2) and notes that ghost cells change that cost (Section 5).
 * These calls predict the same quantity ahead of time: for a tile of edge^3 cells, the
 * blocks it will hold over the next steps.  Summed over tiles, the prediction sizes
 * the block pools of a captured step sequence (vl_translate_opts.capacity).  Nothing
 * here reads or writes f.
 *
 * Tiles: edge^3 cells (the last tile of a dimension may be shorter), numbered x
 * fastest; vl_tile_count gives their number (-1 for bad arguments).
 *
 * vl_tile_features writes, per tile, VL_MLP_NIN float32 features (device buffer
 * [ntiles][VL_MLP_NIN]): log(1+A), log(1+U), log(1+mean n), mean V_x, mean V_y, mean V_z,
 * mean v_th, max |grad n| / n, where A = blocks present in the tile, U = blocks of the
 * tile in the next step's 27-cell union, n, V and v_th = sqrt((Pxx+Pyy+Pzz)/(3n)) are the
 * per-cell moments of vl_moments (V and v_th taken as 0 where n = 0), means over the
 * tile's cells, and grad n by periodic central differences.  union_blocks (device
 * [ntiles]) receives U.  Synchronises the grid's stream; needs a state (VL_ESTATE).
 * Errors: VL_EINVAL (edge outside 1..64, null pointer), VL_ENOMEM, VL_ECUDA.
 *
 * vl_cost_targets: from union_trace (device [nsnap][ntiles], U of consecutive states)
 * the regression targets targets[t][i] = log(1 + max_{0<=j<horizon} U[t+j][i]) for
 * t = 0 .. nsnap-horizon (device).  Errors: VL_EINVAL (nsnap < horizon, horizon < 1).
 *
 * The model: y = b3 + w3 . relu(W2 relu(W1 x + b1) + b2), float32, parameters in one
 * device array of VL_MLP_NPARAM floats laid out W1[64][8] (row = hidden unit), b1[64],
 * W2[64][64], b2[64], w3[64], b3.  Loss L = (1/n) sum_s (y_s - t_s)^2.
 * vl_mlp_forward: y[s] for n samples x[n][8] (device).
 * vl_mlp_gradient: dL/dparams into grad (device, VL_MLP_NPARAM) and L into *loss
 *   (device double), sums over samples in a fixed order in FP64 (reproducible).
 * vl_mlp_train_step: one full-batch Adam step (beta1 VL_MLP_BETA1, beta2 VL_MLP_BETA2,
 *   eps VL_MLP_EPS, bias-corrected; step counts from 1) on params with the moment
 *   arrays adam_m, adam_v (device, VL_MLP_NPARAM each, zero before step 1); *loss
 *   (device, optional) receives L before the update.
 * Both take a caller-provided device workspace, 256-byte aligned, of at least
 * vl_mlp_workspace_bytes(n) bytes, and allocate nothing.
 * vl_mlp_capacity: ceil((1 + margin) * sum_i max(exp(y_i) - 1, 0)) over the tiles'
 *   predictions into *capacity (host); workspace of at least 256*ceil(4*ntiles/256) + 8
 *   bytes.  Synchronises `stream`.
 * All calls queue work on `stream` (cudaStream_t of the current device; NULL = legacy
 * default stream).  Errors: VL_EINVAL (null pointer, n < 0, small or misaligned
 * workspace, step < 1), VL_ECUDA. */
#define VL_MLP_NIN 8
#define VL_MLP_NHIDDEN 64
#define VL_MLP_NPARAM \
    (VL_MLP_NHIDDEN * VL_MLP_NIN + VL_MLP_NHIDDEN * VL_MLP_NHIDDEN + 3 * VL_MLP_NHIDDEN + 1) /* 4801 */
#define VL_MLP_BETA1 0.9f
#define VL_MLP_BETA2 0.999f
#define VL_MLP_EPS 1e-8f
int64_t vl_tile_count(const vl_space_desc* space, int edge);
vl_status vl_tile_features(vl_grid* grid, int edge, float* features, float* union_blocks);
vl_status vl_cost_targets(const float* union_trace, int nsnap, int64_t ntiles, int horizon,
                          float* targets, void* stream);
vl_status vl_mlp_forward(const float* params, const float* x, int64_t n, float* y, void* stream);
size_t vl_mlp_workspace_bytes(int64_t n);
vl_status vl_mlp_gradient(const float* params, const float* x, const float* t, int64_t n,
                          void* workspace, size_t workspace_bytes, float* grad, double* loss,
                          void* stream);
vl_status vl_mlp_train_step(float* params, float* adam_m, float* adam_v, const float* x,
                            const float* t, int64_t n, int step, float lr, void* workspace,
                            size_t workspace_bytes, double* loss, void* stream);
vl_status vl_mlp_capacity(const float* params, const float* features, int64_t ntiles,
                          double margin, void* workspace, size_t workspace_bytes,
                          int64_t* capacity, void* stream);

const char* vl_status_str(vl_status status);
const char* vl_last_error(const vl_grid* grid);

#ifdef __cplusplus
}
#endif
#endif /* VLASOV_H */
