// api.cu -- the C ABI of libvlgt (declared in include/vlasov.h): argument checks,
// device memory through the caller's allocator, and the per-step orchestration of the
// translation (union -> index -> sweeps -> sparsity rule).
#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>
#include <cmath>
#include <cstring>
#include <new>
#include <string>

#include "grid.h"

namespace vlgt {

void* Grid::alloc(size_t bytes)
{
    if (bytes == 0) bytes = 256;
    bytes = (bytes + 255) & ~(size_t)255;
    if (dev.alloc) return dev.alloc(bytes, dev.ctx);
    void* p = nullptr;
    if (cudaMalloc(&p, bytes) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return p;
}

void Grid::release(void* p)
{
    if (!p) return;
    if (dev.free) dev.free(p, dev.ctx);
    else cudaFree(p);
}

static std::atomic<int64_t> g_launches{0};
void note_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
int64_t launch_count() { return g_launches.load(std::memory_order_relaxed); }

vl_status fail(Grid* g, vl_status st, const std::string& msg)
{
    if (g) g->last_error = msg;
    return st;
}

vl_status cuda_fail(Grid* g, cudaError_t e, const char* what)
{
    cudaGetLastError();
    return fail(g, VL_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

}  // namespace vlgt

using namespace vlgt;

namespace {

thread_local std::string g_create_error;

struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev)
    {
        cudaGetDevice(&prev);
        if (prev != dev) cudaSetDevice(dev);
    }
    ~DeviceGuard()
    {
        if (prev >= 0) cudaSetDevice(prev);
    }
};

vl_status parse_order(const char* order, int out[3])
{
    if (!order || std::strlen(order) != 3) return VL_EINVAL;
    int seen[3] = {0, 0, 0};
    for (int j = 0; j < 3; j++) {
        int d = order[j] == 'x' ? 0 : order[j] == 'y' ? 1 : order[j] == 'z' ? 2 : -1;
        if (d < 0 || seen[d]) return VL_EINVAL;
        seen[d] = 1;
        out[j] = d;
    }
    return VL_OK;
}

}  // namespace

extern "C" {

void vl_translate_opts_default(vl_translate_opts* o)
{
    if (!o) return;
    std::memset(o, 0, sizeof(*o));
    o->form = VL_FORM_FUSED;
    o->limiter = 1;
    o->ghost = 3;
}

const char* vl_status_str(vl_status s)
{
    switch (s) {
    case VL_OK: return "VL_OK";
    case VL_EINVAL: return "VL_EINVAL";
    case VL_ENOMEM: return "VL_ENOMEM";
    case VL_ECFL: return "VL_ECFL";
    case VL_ECAPACITY: return "VL_ECAPACITY";
    case VL_ETIMEOUT: return "VL_ETIMEOUT";
    case VL_ECUDA: return "VL_ECUDA";
    case VL_ESTATE: return "VL_ESTATE";
    }
    return "VL_UNKNOWN";
}

const char* vl_last_error(const vl_grid* grid)
{
    if (!grid) return g_create_error.c_str();
    return reinterpret_cast<const Grid*>(grid)->last_error.c_str();
}

vl_status vl_grid_create(const vl_space_desc* space, const vl_vmesh_desc* vmesh,
                         double sparsity_threshold, vl_storage storage, const vl_device* device,
                         vl_grid** out)
{
    g_create_error.clear();
    if (!space || !vmesh || !out) {
        g_create_error = "vl_grid_create: null pointer";
        return VL_EINVAL;
    }
    *out = nullptr;
    for (int d = 0; d < 3; d++) {
        if (space->n[d] <= 0 || !(space->dx[d] > 0.0) || vmesh->nv[d] <= 0 || !(vmesh->dv[d] > 0.0)) {
            g_create_error = "vl_grid_create: extents and cell sizes must be positive";
            return VL_EINVAL;
        }
        if (vmesh->block[d] != 4 || vmesh->nv[d] % 4 != 0) {
            g_create_error = "vl_grid_create: velocity blocks must be 4x4x4 and divide the mesh";
            return VL_EINVAL;
        }
    }
    int64_t nb = (int64_t)(vmesh->nv[0] / 4) * (vmesh->nv[1] / 4) * (vmesh->nv[2] / 4);
    if (nb > 65536) {
        g_create_error = "vl_grid_create: more than 65536 velocity blocks";
        return VL_EINVAL;
    }
    int64_t N = (int64_t)space->n[0] * space->n[1] * space->n[2];
    if (N >= (int64_t)1 << 31) {
        g_create_error = "vl_grid_create: more than 2^31 spatial cells";
        return VL_EINVAL;
    }
    if (storage != VL_STORE_F32) {
        g_create_error = "vl_grid_create: only VL_STORE_F32 is implemented";
        return VL_EINVAL;
    }
    if (!(sparsity_threshold >= 0.0) || !std::isfinite(sparsity_threshold)) {
        g_create_error = "vl_grid_create: the sparsity threshold must be finite and >= 0";
        return VL_EINVAL;
    }
    Grid* g = new (std::nothrow) Grid();
    if (!g) {
        g_create_error = "vl_grid_create: out of host memory";
        return VL_ENOMEM;
    }
    g->space = *space;
    g->vmesh = *vmesh;
    g->threshold = sparsity_threshold;
    g->storage = storage;
    if (device) g->dev = *device;
    else std::memset(&g->dev, 0, sizeof(g->dev));
    g->stream = (cudaStream_t)g->dev.stream;
    DeviceGuard dg(g->dev.device);
    GridGeom& G = g->geom;
    for (int d = 0; d < 3; d++) G.n[d] = space->n[d];
    G.W = (space->n[0] + 63) / 64;
    G.R = (int64_t)space->n[1] * space->n[2];
    G.RW = G.R * G.W;
    G.N = N;
    G.nb = (int)nb;
    G.nbx = vmesh->nv[0] / 4;
    G.nby = vmesh->nv[1] / 4;
    vl_status st = VL_OK;
    for (int i = 0; i < 2 && st == VL_OK; i++) st = layout_alloc_meta(g, g->lay[i]);
    if (st == VL_OK) {
        g->counters = (StepCounters*)g->alloc(sizeof(StepCounters));
        g->item_cnt = (uint32_t*)g->alloc((size_t)nb * 4);
        g->item_base = (int64_t*)g->alloc(((size_t)nb + 1) * 8);
        if (!g->counters || !g->item_cnt || !g->item_base) st = fail(g, VL_ENOMEM, "vl_grid_create: allocation failed");
    }
    const int nvmax = std::max(vmesh->nv[0], std::max(vmesh->nv[1], vmesh->nv[2]));
    if (st == VL_OK) {
        g->ctab = (float4*)g->alloc((size_t)6 * nvmax * sizeof(float4));
        if (!g->ctab) st = fail(g, VL_ENOMEM, "vl_grid_create: allocation failed");
    }
    if (st == VL_OK) {
        cudaError_t e = cudaMallocHost((void**)&g->counters_host, sizeof(StepCounters));
        if (e == cudaSuccess) e = cudaMallocHost((void**)&g->host_scalar, 64);
        if (e == cudaSuccess) e = cudaMallocHost((void**)&g->ctab_host, (size_t)6 * nvmax * sizeof(float4));
        if (e != cudaSuccess) st = cuda_fail(g, e, "vl_grid_create: pinned host memory");
    }
    if (st == VL_OK) {
        cudaError_t e = cudaStreamSynchronize(g->stream);
        if (e != cudaSuccess) st = cuda_fail(g, e, "vl_grid_create");
    }
    if (st != VL_OK) {
        g_create_error = g->last_error;
        vl_grid_destroy(reinterpret_cast<vl_grid*>(g));
        return st;
    }
    g->stats.mass = NAN;
    *out = reinterpret_cast<vl_grid*>(g);
    return VL_OK;
}

vl_status vl_grid_destroy(vl_grid* grid)
{
    if (!grid) return VL_OK;
    Grid* g = reinterpret_cast<Grid*>(grid);
    DeviceGuard dg(g->dev.device);
    cudaStreamSynchronize(g->stream);
    for (int i = 0; i < 2; i++) layout_free(g, g->lay[i]);
    g->release(g->counters);
    g->release(g->item_cnt);
    g->release(g->item_base);
    g->release(g->tile_flags);
    g->release(g->tile_pos);
    g->release(g->items);
    g->release(g->item_mass);
    if (g->ev_sweep0) cudaEventDestroy(g->ev_sweep0);
    if (g->ev_sweep1) cudaEventDestroy(g->ev_sweep1);
    g->release(g->ctab);
    if (g->ctab_host) cudaFreeHost(g->ctab_host);
    if (g->counters_host) cudaFreeHost(g->counters_host);
    if (g->host_scalar) cudaFreeHost(g->host_scalar);
    delete g;
    return VL_OK;
}

vl_status vl_set_blocks(vl_grid* grid, int64_t nblocks, const int64_t* cell_offsets,
                        const uint16_t* block_ids, const float* values, int on_device)
{
    if (!grid) return VL_EINVAL;
    Grid* g = reinterpret_cast<Grid*>(grid);
    DeviceGuard dg(g->dev.device);
    vl_status st = set_blocks(g, nblocks, cell_offsets, block_ids, values, on_device);
    if (st == VL_OK) g->stats.mass = NAN;
    return st;
}

vl_status vl_get_block_count(vl_grid* grid, int64_t* nblocks)
{
    if (!grid || !nblocks) return VL_EINVAL;
    Grid* g = reinterpret_cast<Grid*>(grid);
    DeviceGuard dg(g->dev.device);
    return get_block_count(g, nblocks);
}

vl_status vl_get_blocks(vl_grid* grid, int64_t capacity, int64_t* cell_offsets,
                        uint16_t* block_ids, float* values, int on_device)
{
    if (!grid) return VL_EINVAL;
    Grid* g = reinterpret_cast<Grid*>(grid);
    DeviceGuard dg(g->dev.device);
    return get_blocks(g, capacity, cell_offsets, block_ids, values, on_device);
}

vl_status vl_get_block_count_window(vl_grid* grid, const int origin[3], const int size[3],
                                    int64_t* nblocks)
{
    if (!grid || !origin || !size || !nblocks) return VL_EINVAL;
    Grid* g = reinterpret_cast<Grid*>(grid);
    DeviceGuard dg(g->dev.device);
    return get_window(g, origin, size, 0, nullptr, nullptr, nullptr, 0, nblocks);
}

vl_status vl_get_blocks_window(vl_grid* grid, const int origin[3], const int size[3],
                               int64_t capacity, int64_t* cell_offsets, uint16_t* block_ids,
                               float* values, int on_device)
{
    if (!grid || !origin || !size || !cell_offsets) return VL_EINVAL;
    Grid* g = reinterpret_cast<Grid*>(grid);
    DeviceGuard dg(g->dev.device);
    return get_window(g, origin, size, capacity, cell_offsets, block_ids, values, on_device, nullptr);
}

vl_status vl_moments(vl_grid* grid, double* out, int on_device)
{
    if (!grid) return VL_EINVAL;
    Grid* g = reinterpret_cast<Grid*>(grid);
    DeviceGuard dg(g->dev.device);
    return moments(g, out, on_device);
}

vl_status vl_mass(vl_grid* grid, double* mass)
{
    if (!grid || !mass) return VL_EINVAL;
    Grid* g = reinterpret_cast<Grid*>(grid);
    DeviceGuard dg(g->dev.device);
    return total_mass(g, mass);
}

vl_status vl_stats(vl_grid* grid, vl_step_stats* stats)
{
    if (!grid || !stats) return VL_EINVAL;
    Grid* g = reinterpret_cast<Grid*>(grid);
    *stats = g->stats;
    return VL_OK;
}

vl_status vl_translate(vl_grid* grid, double dt, const char* order, int nsteps,
                       const vl_translate_opts* opts_in)
{
    if (!grid) return VL_EINVAL;
    Grid* g = reinterpret_cast<Grid*>(grid);
    DeviceGuard dg(g->dev.device);
    vl_translate_opts opts;
    if (opts_in) opts = *opts_in;
    else vl_translate_opts_default(&opts);
    StepArgs a;
    if (parse_order(order, a.order) != VL_OK)
        return fail(g, VL_EINVAL, "vl_translate: order must be a permutation of \"xyz\"");
    if (nsteps < 0 || !std::isfinite(dt) || dt < 0.0)
        return fail(g, VL_EINVAL, "vl_translate: dt must be finite and >= 0, nsteps >= 0");
    if (opts.form != VL_FORM_FUSED && opts.form != VL_FORM_3PASS && opts.form != VL_FORM_AUTO)
        return fail(g, VL_EINVAL, "vl_translate: unknown form");
    if (opts.ghost != 3)
        return fail(g, VL_EINVAL, "vl_translate: only the exact ghost depth 3 (GT3) is implemented");
    if (!g->has_state) return fail(g, VL_ESTATE, "vl_translate: no state (call vl_set_blocks first)");
    // Section 2.1: dt keeps every velocity cell within one face neighbour per sweep
    for (int d = 0; d < 3; d++) {
        double lo = std::fabs(g->vmesh.vmin[d] + 0.5 * g->vmesh.dv[d]);
        double hi = std::fabs(g->vmesh.vmin[d] + (g->vmesh.nv[d] - 0.5) * g->vmesh.dv[d]);
        double c = (lo > hi ? lo : hi) * dt / g->space.dx[d];
        if (c > 1.0)
            return fail(g, VL_ECFL, "vl_translate: max |v_d| dt / dx_d = " + std::to_string(c) + " > 1");
        a.c_scale[d] = dt / g->space.dx[d];
    }
    // per-velocity-cell sweep constants (Courant number c = v_d dt / dx_d at the cell
    // centre, Section 2.1), computed in FP64 once per dt and rounded to FP32
    const int nvmax = std::max(g->vmesh.nv[0], std::max(g->vmesh.nv[1], g->vmesh.nv[2]));
    if (g->ctab_dt != dt) {
        cudaStreamSynchronize(g->stream);
        for (int d = 0; d < 3; d++)
            for (int i = 0; i < nvmax; i++) {
                double c = i < g->vmesh.nv[d]
                               ? (g->vmesh.vmin[d] + (i + 0.5) * g->vmesh.dv[d]) * dt / g->space.dx[d]
                               : 0.0;
                WalkConst w = walk_const(c);
                SweepConst k = sweep_const(c);
                g->ctab_host[d * nvmax + i] = make_float4(w.g, w.A, w.B, (float)w.up);
                g->ctab_host[3 * nvmax + d * nvmax + i] = make_float4(k.g, k.A, k.B, (float)k.up);
            }
        cudaMemcpyAsync(g->ctab, g->ctab_host, (size_t)6 * nvmax * sizeof(float4), cudaMemcpyHostToDevice,
                        g->stream);
        g->ctab_dt = dt;
    }
    a.walk = g->ctab;
    a.sweep = g->ctab + 3 * nvmax;
    a.nvmax = nvmax;
    a.limiter = opts.limiter ? 1 : 0;
    a.tile[0] = opts.tile[0];
    a.tile[1] = opts.tile[1];
    const bool fused = opts.form != VL_FORM_3PASS;

    vl_step_stats S{};
    S.mass_before = g->stats.mass;
    cudaEvent_t e0, e1, ei, ep;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    cudaEventCreate(&ei);
    cudaEventCreate(&ep);
    if (!g->ev_sweep0) {
        cudaEventCreate(&g->ev_sweep0);
        cudaEventCreate(&g->ev_sweep1);
    }
    float total_ms = 0.0f, sweep_ms = 0.0f, index_ms = 0.0f, prune_ms = 0.0f;
    const int64_t launches0 = launch_count();
    vl_status st = VL_OK;
    for (int step = 0; step < nsteps && st == VL_OK; step++) {
        Layout& A = g->lay[g->cur];
        Layout& B = g->lay[1 - g->cur];
        cudaEventRecord(e0, g->stream);
        cudaMemsetAsync(g->counters, 0, sizeof(StepCounters), g->stream);
        launch_union(g, A, B);
        int64_t total = 0;
        st = layout_index(g, B, &total);
        if (st != VL_OK) break;
        st = layout_ensure_pool(g, B, std::max<int64_t>(total, 1));
        if (st != VL_OK) break;
        cudaMemsetAsync(B.keepq, 0, (size_t)std::max<int64_t>(total, 1) * 4, g->stream);
        st = fused ? run_fused(g, a) : run_3pass(g, a);
        if (st != VL_OK) break;
        cudaEventRecord(ep, g->stream);
        launch_pack_keep(g, B);
        cudaEventRecord(e1, g->stream);
        cudaMemcpyAsync(g->counters_host, g->counters, sizeof(StepCounters), cudaMemcpyDeviceToHost,
                        g->stream);
        cudaError_t e = cudaStreamSynchronize(g->stream);
        if (e != cudaSuccess) {
            st = cuda_fail(g, e, "vl_translate step");
            break;
        }
        float ms = 0.0f;
        cudaEventElapsedTime(&ms, e0, e1);
        total_ms += ms;
        cudaEventElapsedTime(&ms, g->ev_sweep0, g->ev_sweep1);
        sweep_ms += ms;
        cudaEventElapsedTime(&ms, e0, g->ev_sweep0);
        index_ms += ms;
        cudaEventElapsedTime(&ms, ep, e1);
        prune_ms += ms;
        const StepCounters& C = *g->counters_host;
        if (C.error) {
            st = fail(g, (C.error & 4) ? VL_ETIMEOUT : VL_ECUDA,
                      "vl_translate: device-side error flag " + std::to_string(C.error) +
                          ((C.error & 4) ? " (a staging barrier wait ran out)" : ""));
            break;
        }
        S.steps++;
        S.union_blocks = total;
        S.blocks = (int64_t)C.kept;
        S.dropped_blocks = (int64_t)C.dropped;
        S.dropped_mass += C.dropped_mass * g->space.dx[0] * g->space.dx[1] * g->space.dx[2] *
                          g->vmesh.dv[0] * g->vmesh.dv[1] * g->vmesh.dv[2];
        S.mass = (C.mass - C.dropped_mass) * g->space.dx[0] * g->space.dx[1] * g->space.dx[2] *
                 g->vmesh.dv[0] * g->vmesh.dv[1] * g->vmesh.dv[2];
        g->cur = 1 - g->cur;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaEventDestroy(ei);
    cudaEventDestroy(ep);
    S.device_ms = total_ms;
    S.sweep_ms = sweep_ms;
    S.index_ms = index_ms;
    S.prune_ms = prune_ms;
    S.launches = launch_count() - launches0;
    if (S.steps > 0) g->stats = S;
    else g->stats.steps = 0;
    if (st == VL_OK && opts.check) {
        cudaError_t e = cudaStreamSynchronize(g->stream);
        if (e != cudaSuccess) st = cuda_fail(g, e, "vl_translate");
    }
    return st;
}

}  // extern "C"
