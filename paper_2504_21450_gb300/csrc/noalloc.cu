// noalloc.cu -- a translation step that allocates no memory.
//
// Some callers cannot allocate device memory: code that runs under a strict memory
// budget owned by another runtime, embedded hosts whose allocator is not reachable from
// this library, or callers that must not touch the device heap between two steps.  For them vl_translate_dense_noalloc runs
// the fused Ghost Translation kernel on caller-provided input and output buffers of a
// dense velocity space, and keeps everything else the kernel needs (its work list,
// layout tables, sweep constants and counters) in one statically sized device array
// below.  Every GPU that loads the library holds that array until the process exits.
#include <cuda_runtime.h>
#include <stdint.h>

#include <cmath>
#include <cstring>
#include <mutex>

#include "grid.h"

namespace {

using namespace vlgt;

constexpr size_t kScratchBytes = VL_NOALLOC_SCRATCH_BYTES;  // the limit promised in vlasov.h
static_assert(kScratchBytes % 256 == 0, "scratch size must keep the 256-byte sub-array alignment");

// The scratch of the allocation-free entry point.  Host code must not take its address
// directly (that is a host-side stand-in, not a device address): setup() asks the
// runtime for the device address once per device.
static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
unsigned char* g_scratch_dev[kMaxDevices] = {};

// Device address of g_scratch on `device` (which must be current); looked up on the
// first call per device.
cudaError_t scratch_address(int device, unsigned char** out)
{
    if (device < 0 || device >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_scratch_dev[device]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_dev[device] = static_cast<unsigned char*>(p);
    }
    *out = g_scratch_dev[device];
    return cudaSuccess;
}

struct ScratchLayout {
    size_t counters, ctab, cnt, base, dense, item_base, items, total;
};

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

ScratchLayout layout_for(int nb, int nvmax, int64_t ntiles)
{
    ScratchLayout L;
    size_t o = 0;
    L.counters = o;
    o = align256(o + sizeof(StepCounters));
    L.ctab = o;
    o = align256(o + (size_t)6 * nvmax * sizeof(float4));
    L.cnt = o;
    o = align256(o + (size_t)nb * 4);
    L.base = o;
    o = align256(o + ((size_t)nb + 1) * 8);
    L.dense = o;
    o = align256(o + (size_t)nb);
    L.item_base = o;
    o = align256(o + ((size_t)nb + 1) * 8);
    L.items = o;
    o = align256(o + (size_t)nb * ntiles * 4);
    L.total = o;
    return L;
}

struct SetupArgs {
    int nb;
    int64_t N;
    int64_t ntiles;
    int nvmax;
    int nv[3];
    double vmin[3], dv[3], cs[3];
    uint32_t* cnt;
    int64_t* base;
    uint8_t* dense;
    int64_t* item_base;
    uint32_t* items;
    float4* ctab;
    StepCounters* ctr;
};

// Fills the dense layout tables, the work list of every (block id, tile) pair, the
// sweep constants and zeroed counters, all inside the static scratch.
__global__ void k_noalloc_setup(SetupArgs A)
{
    const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t nthreads = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = tid; i < (int64_t)A.nb * A.ntiles; i += nthreads)
        A.items[i] = (uint32_t)(i % A.ntiles);
    for (int64_t b = tid; b <= A.nb; b += nthreads) {
        A.item_base[b] = b * A.ntiles;
        A.base[b] = b * A.N;
        if (b < A.nb) {
            A.cnt[b] = (uint32_t)A.N;
            A.dense[b] = 3;
        }
    }
    for (int64_t i = tid; i < 3 * (int64_t)A.nvmax; i += nthreads) {
        const int d = (int)(i / A.nvmax), iv = (int)(i % A.nvmax);
        const double c = iv < A.nv[d] ? (A.vmin[d] + (iv + 0.5) * A.dv[d]) * A.cs[d] : 0.0;
        const WalkConst w = walk_const(c);
        const SweepConst k = sweep_const(c);
        A.ctab[i] = make_float4(w.g, w.A, w.B, (float)w.up);
        A.ctab[3 * A.nvmax + i] = make_float4(k.g, k.A, k.B, (float)k.up);
    }
    if (tid == 0) {
        A.ctr->mass = 0.0;
        A.ctr->dropped_mass = 0.0;
        A.ctr->kept = 0;
        A.ctr->dropped = 0;
        A.ctr->work_next = 0;
        A.ctr->error = 0;
        A.ctr->done = 0;
        A.ctr->needed = 0;
    }
}

__global__ void k_noalloc_mass(const StepCounters* ctr, double volume, double* mass_out)
{
    if (threadIdx.x == 0 && blockIdx.x == 0) *mass_out = ctr->mass * volume;
}

}  // namespace

extern "C" vl_status vl_translate_dense_noalloc(const vl_space_desc* space,
                                                const vl_vmesh_desc* vmesh, double dt,
                                                const char* order, int limiter, const float* f_in,
                                                float* f_out, double* mass_out, void* stream)
{
    if (!space || !vmesh || !order || !f_in || !f_out || !mass_out) return VL_EINVAL;
    int ord[3];
    {
        int seen[3] = {0, 0, 0};
        if (std::strlen(order) != 3) return VL_EINVAL;
        for (int j = 0; j < 3; j++) {
            int d = order[j] == 'x' ? 0 : order[j] == 'y' ? 1 : order[j] == 'z' ? 2 : -1;
            if (d < 0 || seen[d]) return VL_EINVAL;
            seen[d] = 1;
            ord[j] = d;
        }
    }
    for (int d = 0; d < 3; d++)
        if (space->n[d] <= 0 || !(space->dx[d] > 0.0) || vmesh->nv[d] <= 0 || vmesh->nv[d] % 4 != 0 ||
            vmesh->block[d] != 4 || !(vmesh->dv[d] > 0.0))
            return VL_EINVAL;
    if (f_in == f_out || !std::isfinite(dt) || dt < 0.0) return VL_EINVAL;
    for (int d = 0; d < 3; d++) {
        double lo = std::fabs(vmesh->vmin[d] + 0.5 * vmesh->dv[d]);
        double hi = std::fabs(vmesh->vmin[d] + (vmesh->nv[d] - 0.5) * vmesh->dv[d]);
        if ((lo > hi ? lo : hi) * dt / space->dx[d] > 1.0) return VL_ECFL;
    }
    GridGeom G;
    G.abort = nullptr;
    for (int d = 0; d < 3; d++) G.n[d] = space->n[d];
    G.W = (space->n[0] + 63) / 64;
    G.R = (int64_t)space->n[1] * space->n[2];
    G.RW = G.R * G.W;
    G.N = (int64_t)space->n[0] * space->n[1] * space->n[2];
    G.nb = (vmesh->nv[0] / 4) * (vmesh->nv[1] / 4) * (vmesh->nv[2] / 4);
    G.nbx = vmesh->nv[0] / 4;
    G.nby = vmesh->nv[1] / 4;
    const int nvmax = std::max(vmesh->nv[0], std::max(vmesh->nv[1], vmesh->nv[2]));
    const int ty = fused_tile_rows(ord);
    const int ntile0 = (G.n[ord[0]] + kFusedTileX - 1) / kFusedTileX;
    const int64_t ntiles = (int64_t)ntile0 * ((G.n[ord[1]] + ty - 1) / ty);
    const ScratchLayout SL = layout_for(G.nb, nvmax, ntiles);
    if (SL.total > kScratchBytes || G.N >= ((int64_t)1 << 31)) return VL_ECAPACITY;

    int device = 0;
    if (cudaGetDevice(&device) != cudaSuccess) return VL_ECUDA;
    unsigned char* scratch = nullptr;
    if (scratch_address(device, &scratch) != cudaSuccess) {
        cudaGetLastError();
        return VL_ECUDA;
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    SetupArgs A;
    A.nb = G.nb;
    A.N = G.N;
    A.ntiles = ntiles;
    A.nvmax = nvmax;
    for (int d = 0; d < 3; d++) {
        A.nv[d] = vmesh->nv[d];
        A.vmin[d] = vmesh->vmin[d];
        A.dv[d] = vmesh->dv[d];
        A.cs[d] = dt / space->dx[d];
    }
    A.cnt = reinterpret_cast<uint32_t*>(scratch + SL.cnt);
    A.base = reinterpret_cast<int64_t*>(scratch + SL.base);
    A.dense = scratch + SL.dense;
    A.item_base = reinterpret_cast<int64_t*>(scratch + SL.item_base);
    A.items = reinterpret_cast<uint32_t*>(scratch + SL.items);
    A.ctab = reinterpret_cast<float4*>(scratch + SL.ctab);
    A.ctr = reinterpret_cast<StepCounters*>(scratch + SL.counters);
    k_noalloc_setup<<<64, 256, 0, s>>>(A);

    LayoutView in{nullptr, nullptr, nullptr, A.cnt, A.base, A.dense, const_cast<float*>(f_in)};
    LayoutView out{nullptr, nullptr, nullptr, A.cnt, A.base, A.dense, f_out};
    vl_status st = launch_fused_dense(G, in, out, ord, limiter ? 1 : 0, A.ctab, nvmax, A.items,
                                      A.item_base, ntile0, A.ctr, device, s);
    if (st != VL_OK) return st;
    const double vol = space->dx[0] * space->dx[1] * space->dx[2] * vmesh->dv[0] * vmesh->dv[1] * vmesh->dv[2];
    k_noalloc_mass<<<1, 32, 0, s>>>(A.ctr, vol, mass_out);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? VL_OK : VL_ECUDA;
}
