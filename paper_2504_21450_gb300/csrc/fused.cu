// fused.cu -- Ghost Translation on one GPU: the three sweeps of a translation step in
// one kernel over a spatial tile plus its ghost halo (paper Section 3).
//
// A work item is (block id b, velocity chunk q, tile column).  The tile spans TX x TY
// cells along the first two sweep axes and the whole periodic extent of the third axis,
// which is streamed plane by plane.  Every plane of the tile plus a halo of 3 cells
// (GT3: the 2-cell stencil plus one face neighbour, Section 3.1) is staged into shared
// memory exactly once with 16-byte cp.async copies (the coalesced ghost update); the
// first sweep then runs on the tile rows widened by the halo along the second axis
// (the paper's active cells of the first sweep), the second sweep on the tile, and the
// third sweep consumes the planes from a 7-deep sliding window that each thread keeps
// in registers, so that no intermediate result goes back to HBM.
//
// Thread layout (256 threads): lane v = tid % 16 is the velocity cell of the chunk;
// first sweep: tid / 16 = halo row (14 rows); second and third sweeps: tid / 16 = tile
// column along axis 0, each thread owning the TY cells of that column.
#include <cuda_runtime.h>
#include <stdint.h>

#include "grid.h"

namespace vlgt {

namespace {

constexpr int TX = 16, TY = 8;
constexpr int NT = 256;
constexpr int NST = 3;                     // pipeline stages of staged planes
constexpr int EX = TX + 2 * kHalo;         // 22
constexpr int EY = TY + 2 * kHalo;         // 14
constexpr int SROW = EX * kChunk + 16;     // padded stage row (floats); 16 mod 32 keeps
constexpr int STAGE = EY * SROW;           // two rows of a warp on distinct banks
constexpr int XROW = TX * kChunk + 16;
constexpr int XBUF = EY * XROW;
constexpr int kSmemBytes = (NST * STAGE + XBUF) * 4 + 2 * TX * TY * 4 + 64;

static_assert(EY * kChunk <= NT, "first-sweep rows must fit the CTA");
static_assert(TX * kChunk == NT, "second-sweep columns must match the CTA");

struct FusedArgs {
    GridGeom G;
    LayoutView in, out;
    int ax[3];           // physical axis of sweep 0, 1, 2 (axis 2 is streamed)
    double cs[3];        // dt / dx of sweep j's axis
    double vmin[3], dv[3];
    float thr;
    int ntile0;          // tiles along sweep axis 0
    const uint32_t* items;
    const int64_t* item_base;  // [nb + 1]
    uint8_t* keepq;
    StepCounters* ctr;
};

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem, int src_bytes)
{
    unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(s), "l"(gmem), "r"(src_bytes)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

__device__ __forceinline__ void to_phys(const int ax[3], int l0, int l1, int l2, int& x, int& y, int& z)
{
    int p[3];
    p[ax[0]] = l0;
    p[ax[1]] = l1;
    p[ax[2]] = l2;
    x = p[0];
    y = p[1];
    z = p[2];
}

template <bool kLim>
__global__ void __launch_bounds__(NT, 2) k_fused(FusedArgs P)
{
    extern __shared__ __align__(16) float smem[];
    float* stage = smem;
    float* xbuf = smem + NST * STAGE;
    int* orank = reinterpret_cast<int*>(xbuf + XBUF);  // [2][TY][TX]
    __shared__ int64_t s_work;

    const GridGeom& G = P.G;
    const int tid = threadIdx.x;
    const int v = tid & 15;
    const int hi = tid >> 4;  // halo row (sweep 0) / tile column (sweeps 1, 2)
    const int n0 = G.n[P.ax[0]], n1 = G.n[P.ax[1]], n2 = G.n[P.ax[2]];
    const int64_t nwork = 4 * P.item_base[G.nb];
    const int nplanes = n2 + 2 * kHalo;

    for (;;) {
        __syncthreads();  // previous item fully done with shared memory
        if (tid == 0) s_work = (int64_t)atomicAdd(&P.ctr->work_next, 1ull);
        __syncthreads();
        const int64_t w = s_work;
        if (w >= nwork) break;

        // decode (b, q, tile): items are grouped by b; within b, q-major then tile
        int lo = 0, hi_b = G.nb;
        while (hi_b - lo > 1) {
            int mid = (lo + hi_b) >> 1;
            if (4 * P.item_base[mid] <= w) lo = mid;
            else hi_b = mid;
        }
        const int b = lo;
        const int64_t mb = P.item_base[b + 1] - P.item_base[b];
        const int64_t wl = w - 4 * P.item_base[b];
        const int q = (int)(wl / mb);
        const uint32_t tile = P.items[P.item_base[b] + (wl % mb)];
        const int t0 = (int)(tile % P.ntile0) * TX;
        const int t1 = (int)(tile / P.ntile0) * TY;
        const int e0 = min(TX, n0 - t0), e1 = min(TY, n1 - t1);

        // per-thread velocity cell (chunk q = vz plane of the block; v = vx + 4 vy)
        const int bcoord[3] = {b % G.nbx, (b / G.nbx) % G.nby, b / (G.nbx * G.nby)};
        const int within[3] = {v & 3, v >> 2, q};
        SweepConst kc[3];
#pragma unroll
        for (int j = 0; j < 3; j++) {
            int d = P.ax[j];
            int iv = bcoord[d] * 4 + within[d];
            kc[j] = sweep_const((P.vmin[d] + (iv + 0.5) * P.dv[d]) * P.cs[j]);
        }
        const int64_t ibase = ((int64_t)P.in.base[b] * 4 + (int64_t)q * P.in.cnt[b]) * kChunk;
        const int64_t obase = ((int64_t)P.out.base[b] * 4 + (int64_t)q * P.out.cnt[b]) * kChunk;
        const int64_t okeep = (int64_t)P.out.base[b];

        auto issue_plane = [&](int it) {
            if (it < nplanes) {
                const int pz = wrapi(it - kHalo, n2);
                float* st = stage + (it % NST) * STAGE;
                for (int cidx = tid; cidx < EX * EY; cidx += NT) {
                    int u1 = cidx / EX, u0 = cidx - u1 * EX;
                    int x, y, z;
                    to_phys(P.ax, wrapi(t0 - kHalo + u0, n0), wrapi(t1 - kHalo + u1, n1), pz, x, y, z);
                    int64_t row = y + (int64_t)G.n[1] * z;
                    int64_t r = cell_rank(P.in, G, b, x, row, true);
                    const float* src = r >= 0 ? P.in.pool + ibase + r * kChunk : P.in.pool;
                    float* dstp = st + u1 * SROW + u0 * kChunk;
                    int nb = r >= 0 ? 16 : 0;
#pragma unroll
                    for (int j = 0; j < 4; j++) cp_async16(dstp + 4 * j, src + 4 * j, nb);
                }
            }
            cp_async_commit();
        };

        Slide<kLim> zs[TY];
#pragma unroll
        for (int j = 0; j < TY; j++) zs[j].reset();
        float msum = 0.0f;
        double mass = 0.0;

#pragma unroll
        for (int it = 0; it < NST - 1; it++) issue_plane(it);

        for (int it = 0; it < nplanes; it++) {
            issue_plane(it + NST - 1);
            // ranks of the output plane (it - 6) in the next layout
            const int k = it - 2 * kHalo;
            if (k >= 0 && tid < TX * TY) {
                int j = tid / TX, i = tid - j * TX;
                int r = -1;
                if (i < e0 && j < e1) {
                    int x, y, z;
                    to_phys(P.ax, t0 + i, t1 + j, k, x, y, z);
                    r = (int)cell_rank(P.out, G, b, x, y + (int64_t)G.n[1] * z, false);
                }
                orank[(it & 1) * TX * TY + tid] = r;
            }
            cp_async_wait<NST - 1>();
            __syncthreads();

            // sweep 0 along axis 0 on all EY halo rows
            const float* st = stage + (it % NST) * STAGE;
            if (hi < EY) {
                Slide<kLim> s;
                s.reset();
                const float* line = st + hi * SROW + v;
                float* xo = xbuf + hi * XROW + v;
#pragma unroll
                for (int u = 0; u < EX; u++) {
                    float res = s.push(line[u * kChunk], kc[0]);
                    if (u >= 2 * kHalo) xo[(u - 2 * kHalo) * kChunk] = res;
                }
            }
            __syncthreads();

            // sweep 1 along axis 1 for tile column `hi`, then sweep 2 (streamed)
            float col[TY];
            {
                Slide<kLim> s;
                s.reset();
                const float* line = xbuf + hi * kChunk + v;
#pragma unroll
                for (int r = 0; r < EY; r++) {
                    float res = s.push(line[r * XROW], kc[1]);
                    if (r >= 2 * kHalo) col[r - 2 * kHalo] = res;
                }
            }
            const int* orow = orank + (it & 1) * TX * TY;
#pragma unroll
            for (int j = 0; j < TY; j++) {
                float res = zs[j].push(col[j], kc[2]);
                if (k >= 0) {
                    int r = orow[j * TX + hi];
                    if (r >= 0) {
                        P.out.pool[obase + (int64_t)r * kChunk + v] = res;
                        msum += res;
                    }
                    unsigned m = __ballot_sync(0xffffffffu, r >= 0 && res >= P.thr);
                    if (r >= 0 && v == 0) {
                        unsigned half = (tid & 16) ? (m >> 16) : (m & 0xffffu);
                        P.keepq[(okeep + r) * 4 + q] = half ? 1 : 0;
                    }
                }
            }
            mass += (double)msum;
            msum = 0.0f;
        }
        cp_async_wait<0>();
        for (int o = 16; o > 0; o >>= 1) mass += __shfl_xor_sync(0xffffffffu, mass, o);
        if ((tid & 31) == 0 && mass != 0.0) atomicAdd(&P.ctr->mass, mass);
    }
}

// ---- work list ------------------------------------------------------------------
struct TileArgs {
    GridGeom G;
    const uint64_t* ubits;
    int ax[3];
    int ntile0, ntile1;
};

__device__ bool row_any(const uint64_t* rowp, int xlo, int xhi)
{
    uint64_t acc = 0;
    for (int w = xlo >> 6; w <= ((xhi - 1) >> 6); w++) {
        uint64_t m = ~0ull;
        if (w == (xlo >> 6)) m &= ~0ull << (xlo & 63);
        if (w == ((xhi - 1) >> 6) && ((xhi - 1) & 63) != 63) m &= (1ull << (((xhi - 1) & 63) + 1)) - 1ull;
        acc |= rowp[w] & m;
    }
    return acc != 0;
}

// flag[b][tile] = 1 when the tile column holds any slot of block id b in the next layout
__global__ void k_tile_flags(TileArgs T, uint32_t* __restrict__ flags)
{
    const GridGeom& G = T.G;
    int64_t ntiles = (int64_t)T.ntile0 * T.ntile1;
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (int64_t)G.nb * ntiles) return;
    int b = (int)(i / ntiles);
    int tile = (int)(i - (int64_t)b * ntiles);
    int lo[3], hi[3];
    lo[T.ax[0]] = (tile % T.ntile0) * TX;
    hi[T.ax[0]] = min(lo[T.ax[0]] + TX, G.n[T.ax[0]]);
    lo[T.ax[1]] = (tile / T.ntile0) * TY;
    hi[T.ax[1]] = min(lo[T.ax[1]] + TY, G.n[T.ax[1]]);
    lo[T.ax[2]] = 0;
    hi[T.ax[2]] = G.n[T.ax[2]];
    const uint64_t* seg = T.ubits + (int64_t)b * G.RW;
    bool any = false;
    for (int z = lo[2]; z < hi[2] && !any; z++)
        for (int y = lo[1]; y < hi[1] && !any; y++)
            any = row_any(seg + ((int64_t)y + (int64_t)G.n[1] * z) * G.W, lo[0], hi[0]);
    flags[i] = any ? 1u : 0u;
}

__global__ void k_tile_items(int64_t ntiles, int nb, const uint32_t* __restrict__ flags,
                             const uint32_t* __restrict__ pos, const int64_t* __restrict__ base,
                             uint32_t* __restrict__ items)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (int64_t)nb * ntiles) return;
    if (!flags[i]) return;
    int b = (int)(i / ntiles);
    items[base[b] + pos[i]] = (uint32_t)(i - (int64_t)b * ntiles);
}

inline int nblk(int64_t n, int t) { return (int)((n + t - 1) / t); }

}  // namespace

vl_status run_fused(Grid* g, const StepArgs& a)
{
    const GridGeom& G = g->geom;
    Layout& A = g->lay[g->cur];
    Layout& B = g->lay[1 - g->cur];
    int ax[3] = {a.order[0], a.order[1], a.order[2]};
    int ntile0 = (G.n[ax[0]] + TX - 1) / TX;
    int ntile1 = (G.n[ax[1]] + TY - 1) / TY;
    int64_t ntiles = (int64_t)ntile0 * ntile1;
    if (ntiles > 0xffffffffLL) return fail(g, VL_EINVAL, "fused form: too many tiles");
    int64_t need = ntiles * G.nb;
    if (need > g->ntiles_alloc) {
        g->release(g->tile_flags);
        g->release(g->tile_pos);
        g->release(g->items);
        g->tile_flags = (uint32_t*)g->alloc((size_t)need * 4);
        g->tile_pos = (uint32_t*)g->alloc((size_t)need * 4);
        g->items = (uint32_t*)g->alloc((size_t)need * 4);
        if (!g->tile_flags || !g->tile_pos || !g->items) {
            g->ntiles_alloc = 0;
            return fail(g, VL_ENOMEM, "fused form: work-list allocation failed");
        }
        g->ntiles_alloc = need;
    }
    TileArgs T;
    T.G = G;
    T.ubits = B.ubits;
    for (int j = 0; j < 3; j++) T.ax[j] = ax[j];
    T.ntile0 = ntile0;
    T.ntile1 = ntile1;
    k_tile_flags<<<nblk(need, 256), 256, 0, g->stream>>>(T, g->tile_flags); note_launch();
    launch_seg_scan(g->tile_flags, g->tile_pos, g->item_cnt, ntiles, G.nb, g->stream);
    launch_base_scan(g->item_cnt, g->item_base, G.nb, g->stream);
    k_tile_items<<<nblk(need, 256), 256, 0, g->stream>>>(ntiles, G.nb, g->tile_flags, g->tile_pos,
                                                           g->item_base, g->items); note_launch();

    FusedArgs P;
    P.G = G;
    P.in = A.view();
    P.out = B.view();
    for (int j = 0; j < 3; j++) {
        P.ax[j] = ax[j];
        P.cs[j] = a.c_scale[ax[j]];
        P.vmin[j] = g->vmesh.vmin[j];
        P.dv[j] = g->vmesh.dv[j];
    }
    P.thr = (float)g->threshold;
    P.ntile0 = ntile0;
    P.items = g->items;
    P.item_base = g->item_base;
    P.keepq = B.keepq;
    P.ctr = g->counters;
    static int configured = 0;
    if (!configured) {
        cudaFuncSetAttribute(k_fused<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemBytes);
        cudaFuncSetAttribute(k_fused<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemBytes);
        configured = 1;
    }
    int nsm = 0;
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, g->dev.device);
    int per_sm = 0;
    if (a.limiter)
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_fused<true>, NT, kSmemBytes);
    else
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_fused<false>, NT, kSmemBytes);
    if (per_sm < 1) per_sm = 1;
    int grid = nsm * per_sm;
    cudaEventRecord(g->ev_sweep0, g->stream);
    if (a.limiter) {
        k_fused<true><<<grid, NT, kSmemBytes, g->stream>>>(P); note_launch();
    }
    else {
        k_fused<false><<<grid, NT, kSmemBytes, g->stream>>>(P); note_launch();
    }
    cudaEventRecord(g->ev_sweep1, g->stream);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(g, e, "fused sweep launch");
    return VL_OK;
}

}  // namespace vlgt
