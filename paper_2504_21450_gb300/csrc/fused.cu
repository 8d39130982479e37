// fused.cu -- Ghost Translation on one GPU: the three sweeps of a translation step in
// one kernel over a spatial tile plus its ghost halo (paper Section 3).
//
// A work item is (block id b, velocity chunk q, tile column).  The tile spans TX x TY
// cells along the first two sweep axes and the whole periodic extent of the third
// axis, which is streamed plane by plane.  Every plane of the tile plus a halo of 3
// cells (GT3: the 2-cell stencil plus one face neighbour, Section 3.1) is staged into
// shared memory exactly once with 16-byte cp.async copies (the single coalesced ghost
// update).  Sweep 0 then runs on all halo rows (the active cells of the first sweep),
// sweep 1 on the tile columns, and sweep 2 consumes the planes through a sliding
// window that each thread keeps in registers, so no intermediate result goes to HBM.
//
// Each sweep walks its line from the upwind side (Walk), so its arithmetic has no
// sign-dependent selects.  When the streamed axis is the velocity chunk's own axis
// (sweep order ending in z, the chunk being a vz plane), every velocity cell of an
// item shares the sign of c along it and the planes are streamed upwind-first too;
// otherwise the streamed sweep uses the sign-generic window (Slide).
//
// Thread roles (512 threads, lane = velocity cell): during sweep 0 the threads of the
// halo rows (22 x 16) run it while the others stage the next planes, compute output
// slots of sparse layouts and write the per-chunk keep flags of the sparsity rule;
// then every thread runs sweep 1 on one segment of a tile column (TY/2 rows) and keeps
// the streamed windows of those cells for sweep 2.
#include <cuda_runtime.h>
#include <stdint.h>

#include <cmath>
#include <type_traits>

#include "grid.h"

namespace vlgt {

namespace {

constexpr int NV = kChunk;   // velocity cells per item (one vz plane of a block)
constexpr int H = kHalo;
constexpr int TX = 16;
constexpr int NT = 512;
constexpr int NST = 3;               // pipeline stages of staged planes
constexpr int EX = TX + 2 * H;       // 22 halo columns
constexpr int SROW = EX * NV + 16;   // padded stage row (values), 16 mod 32
constexpr int XROW = TX * NV + 16;   // padded sweep-0 output row

template <int TY_, int ES_ = 4>
struct Shape {
    static constexpr int TY = TY_;
    static constexpr int ES = ES_;            // bytes per staged value (storage type)
    static constexpr int EY = TY + 2 * H;
    static constexpr int NX = EY * NV;        // threads of sweep 0
    static constexpr int NLD = NT - NX;       // threads staging planes meanwhile
    static constexpr int NH = NT / (TX * NV); // sweep-1 segments per tile column
    static constexpr int L = TY / NH;         // tile rows per sweep-1 segment
    static constexpr int STAGE = EY * SROW;
    static constexpr int XBUF = EY * XROW;
    static constexpr int TABS = 2 * EX + 2 * EY;
    // 16-bit storage adds the chunk scales of the staged cells ([NST][EY][EX] floats)
    static constexpr int SCALES = ES < 4 ? NST * EY * EX : 0;
    static constexpr int SMEM = NST * STAGE * ES + 2 * XBUF * 4 + TABS * 4 + 4 * TX * TY * 4 + 3 * 16 * 4 +
                                SCALES * 4 + 64;
    static_assert(NX < NT, "sweep-0 rows must leave threads to stage planes");
    static_assert(NH * TX * NV == NT && NH * L == TY, "sweep-1 segments must tile the CTA");
};

struct FusedArgs {
    GridGeom G;
    LayoutView in, out;
    int ax[3];           // physical axis of sweep 0, 1, 2 (axis 2 is streamed)
    int64_t stride[3];   // cell-index stride of each physical axis (1, nx, nx*ny)
    const float4* walk;   // [3][nvmax] WalkConst (g, A, B, up) per axis and velocity index
    const float4* sweep;  // [3][nvmax] SweepConst (g, A, B, up)
    int nvmax;
    float thr;
    int ntile0;          // tiles along sweep axis 0
    const uint32_t* items;
    const int64_t* item_base;  // [nb + 1]
    uint8_t* keepq;
    StepCounters* ctr;
    int report_late;     // testing hook: a staging wait that is not complete at its first
                         // poll is reported as overdue (VL_ETIMEOUT), then waited for
    uint64_t* cta_done;  // optional [gridDim.x]: %globaltimer when the CTA ran out of work
    int gt_k;            // ghost depth of GT-k, 1..3 (3: exact)
};

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem, int src_bytes)
{
    unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(s), "l"(gmem), "r"(src_bytes)
                 : "memory");
}
// 4-byte copy global -> shared (the chunk scale of a staged cell); src_bytes = 0 writes 0
__device__ __forceinline__ void cp_async4(void* smem, const void* gmem, int src_bytes)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"((unsigned)__cvta_generic_to_shared(smem)),
                 "l"(gmem), "r"(src_bytes)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

// x and row contributions of coordinate c along physical axis d
__device__ __forceinline__ int xpart(int d, int c) { return d == 0 ? c : 0; }
__device__ __forceinline__ int rpart(int d, int c, int ny) { return d == 1 ? c : (d == 2 ? c * ny : 0); }

__device__ __forceinline__ unsigned smem_u32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, unsigned bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, unsigned parity)
{
    unsigned ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ bool mbar_test_wait(uint64_t* bar, unsigned parity)
{
    unsigned ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ uint64_t globaltimer_ns()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;\n" : "=l"(t));
    return t;
}
__device__ __forceinline__ void mbar_add_tx(uint64_t* bar, unsigned bytes)
{
    asm volatile("mbarrier.expect_tx.relaxed.cta.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(smem_u32(bar)) : "memory");
}
// 1D bulk copy global -> shared (TMA), completion counted on an mbarrier
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, unsigned bytes, uint64_t* bar)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

// Bounds of a staging wait before the kernel gives up and flags VL_ETIMEOUT: one second
// of device time (a plane is a few tens of kB, staged in microseconds), and a poll count
// as a second limit.  Reaching either means a fault upstream.
constexpr unsigned kMaxPolls = 1u << 24;
constexpr uint64_t kWaitNs = 1000000000ull;

template <int TY, bool kLim, bool kZUni, int kCodec, bool kRed = false>
__global__ void __launch_bounds__(NT, 1) k_fused(FusedArgs P)
{
    using C = Codec<kCodec>;
    using T = typename C::T;
    using S = Shape<TY, (int)sizeof(T)>;
    constexpr int PC = NV * (int)sizeof(T) / 16;  // 16-byte pieces per staged cell
    constexpr int EY = S::EY;
    constexpr int NLD = S::NLD, L = S::L;
    extern __shared__ __align__(16) float smem[];
    T* stage = reinterpret_cast<T*>(smem);
    float* xbuf = reinterpret_cast<float*>(stage + NST * S::STAGE);
    int* px0 = reinterpret_cast<int*>(xbuf + 2 * S::XBUF);  // xbuf: [2] planes
    int* pr0 = px0 + EX;
    int* px1 = pr0 + EX;
    int* pr1 = px1 + EY;
    int* orank = pr1 + EY;                                           // [4][TY][TX]
    unsigned* kb = reinterpret_cast<unsigned*>(orank + 4 * TX * TY);  // [3][16 warps]
    float* isc = reinterpret_cast<float*>(kb + 3 * 16);               // [NST][EY][EX] (16-bit)
    __shared__ int64_t s_work;
    __shared__ __align__(8) uint64_t s_bar[NST];  // staging barriers of the bulk copies
    __shared__ int s_run[EX][3];                  // contiguous runs of a halo row: u0, x, len
    __shared__ int s_nrun;
    __shared__ int s_abort[2];  // a staging wait of an even / odd plane ran out: stop and leave

    const GridGeom& G = P.G;
    if (aborted(G.abort)) return;
    const int tid = threadIdx.x;
    const int v = tid & 15;
    const int hi = tid >> 4;
    const int lane = tid & 31, warp = tid >> 5;
    const int a0 = P.ax[0], a1 = P.ax[1], a2 = P.ax[2];
    const int n0 = G.n[a0], n1 = G.n[a1], n2 = G.n[a2];
    const int ny = G.n[1];
    const int64_t nwork = 4 * P.item_base[G.nb];
    // The streamed window returns the new average of the plane 2 (Walk) or 3 (Slide)
    // positions behind the one pushed, and the first pushed plane is 3 before the
    // first cell: outputs start at step FIRST and cover steps FIRST .. n2+FIRST-1.
    constexpr int FIRST = H + (kZUni ? 2 : 3);
    const int nsteps = n2 + FIRST;  // planes streamed per item
    const bool loader = tid >= S::NX;
    const int ltid = tid - S::NX;
    const int ci = hi & (TX - 1);       // sweep-1 segment: tile column ci,
    const int j0 = (tid / (TX * NV)) * L;  // rows j0 .. j0+L-1

    if (tid == 0) {
        for (int k = 0; k < NST; k++) mbar_init(&s_bar[k], 1);
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
        s_abort[0] = s_abort[1] = 0;
    }
    unsigned gstep = 0;  // planes staged by this CTA so far (barrier phases)

    for (;;) {
        __syncthreads();
        if (tid == 0) s_work = (int64_t)atomicAdd(&P.ctr->work_next, 1ull);
        __syncthreads();
        const int64_t w = s_work;
        if (w >= nwork || s_abort[0] || s_abort[1]) break;

        // ---- decode (b, q, tile); items are grouped by b, q-major then tile --------
        int lo = 0, hb = G.nb;
        while (hb - lo > 1) {
            int mid = (lo + hb) >> 1;
            if (4 * P.item_base[mid] <= w) lo = mid;
            else hb = mid;
        }
        const int b = lo;
        const int64_t mb = P.item_base[b + 1] - P.item_base[b];
        const int64_t wl = w - 4 * P.item_base[b];
        const int q = (int)(wl / mb);
        const uint32_t tile = P.items[P.item_base[b] + (wl % mb)];
        const int t0 = (int)(tile % P.ntile0) * TX;
        const int t1 = (int)(tile / P.ntile0) * TY;
        const int e0 = min(TX, n0 - t0), e1 = min(TY, n1 - t1);
        const bool dense_in = (P.in.dense[b] & 3) == 3;
        const bool dense_out = (P.out.dense[b] & 1) != 0;
        const bool bulk = dense_in && a0 == 0;  // halo rows are contiguous runs in HBM
        const bool sbulk = !dense_in && a0 == 0;  // sparse rows: runs of present cells
        const bool full = e0 == TX && e1 == TY;
        // GT-k (Section 3.2): sweep 0 runs on the halo rows within k of the tile along
        // axis 1 (with k = 3, every row a sweep-1 stencil of the tile reads).  In the
        // reduced variants (kRed: k = 1, 2) the other rows walk with c = 0, which
        // returns every value unchanged (no outflow, and a - (+-0) + (+-0) = a), so
        // they enter sweep 1 with their pre-step values
        const bool x_active = hi - H >= -P.gt_k && hi - H < e1 + P.gt_k;
        const int64_t ibase = ((int64_t)P.in.base[b] * 4 + (int64_t)q * P.in.cnt[b]) * NV;
        const int64_t obase = ((int64_t)P.out.base[b] * 4 + (int64_t)q * P.out.cnt[b]) * NV;
        const int64_t okeep = (int64_t)P.out.base[b];
        const T* ipool = static_cast<const T*>(P.in.pool);
        T* opool = static_cast<T*>(P.out.pool);

        // contiguous runs of a halo row along axis 0 (split at the periodic wrap)
        if (tid == 0 && (bulk || sbulk)) {
            int u0 = 0, nr = 0;
            while (u0 < EX) {
                const int x = wrapi(t0 - H + u0, n0);
                const int len = min(EX - u0, n0 - x);
                s_run[nr][0] = u0;
                s_run[nr][1] = x;
                s_run[nr][2] = len;
                nr++;
                u0 += len;
            }
            s_nrun = nr;
        }
        // wrapped halo coordinates of sweep axes 0 and 1, split into x and row parts
        if (tid < EX) {
            int c = wrapi(t0 - H + tid, n0);
            px0[tid] = xpart(a0, c);
            pr0[tid] = rpart(a0, c, ny);
        } else if (tid >= 32 && tid < 32 + EY) {
            int u = tid - 32;
            int c = wrapi(t1 - H + u, n1);
            px1[u] = xpart(a1, c);
            pr1[u] = rpart(a1, c, ny);
        }

        // sweep constants of this thread's velocity cell (chunk q = vz plane, v = vx + 4 vy)
        const int bc[3] = {b % G.nbx, (b / G.nbx) % G.nby, b / (G.nbx * G.nby)};
        const int wi[3] = {v & 3, v >> 2, q};
        WalkConst kw[3];
        SweepConst ks2;
#pragma unroll
        for (int j = 0; j < 3; j++) {
            const int d = P.ax[j];
            const int iv = (d == 0 ? bc[0] : d == 1 ? bc[1] : bc[2]) * 4 + (d == 0 ? wi[0] : d == 1 ? wi[1] : wi[2]);
            const float4 c4 = P.walk[d * P.nvmax + iv];
            kw[j] = WalkConst{c4.x, c4.y, c4.z, c4.w != 0.0f ? 1 : 0};
            if (j == 2) {
                const float4 s4 = P.sweep[d * P.nvmax + iv];
                ks2 = SweepConst{s4.x, s4.y, s4.z, s4.w != 0.0f ? 1 : 0};
            }
        }
        const WalkConst kx = (!kRed || x_active) ? kw[0] : WalkConst{0.0f, 0.0f, 0.0f, kw[0].up};
        const bool zup = kw[2].up != 0;  // uniform over the item when kZUni
        // streamed plane of step s and the output plane it completes
        auto plane_of = [&](int s) { return kZUni ? (zup ? s - H : n2 + 2 - s) : s - H; };
        auto out_of = [&](int s) { return kZUni ? (zup ? s - 5 : n2 + 4 - s) : s - 6; };
        __syncthreads();  // tables ready

        // ---- staging of plane s into stage s % NST --------------------------------
        auto issue_plane = [&](int s) {
            if (s < nsteps) {
                const int pz = wrapi(plane_of(s), n2);
                const int x2 = xpart(a2, pz), r2 = rpart(a2, pz, ny);
                T* st = stage + (s % NST) * S::STAGE;
                if (bulk) {
                    // one lane expects the plane's bytes, then lane u1 copies halo row u1
                    // as one bulk copy per contiguous run
                    uint64_t* bar = &s_bar[(gstep + s) % NST];
                    if (ltid == 0) {
                        asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
                        mbar_expect_tx(bar, (unsigned)(EX * EY * NV * sizeof(T)));
                    }
                    __syncwarp();
                    if (ltid < EY) {
                        asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
                        const int64_t row = (int64_t)pr1[ltid] + r2;
                        const T* src = ipool + ibase + row * G.n[0] * NV;
                        T* dst = st + ltid * SROW;
                        for (int k = 0; k < s_nrun; k++)
                            bulk_g2s(dst + s_run[k][0] * NV, src + s_run[k][1] * NV,
                                     (unsigned)(s_run[k][2] * NV * sizeof(T)), bar);
                    }
                } else if (sbulk) {
                    // lane u1 stages halo row u1.  The row's bitmap words are read once
                    // (a run spans at most two); each run of present cells, whose slots are
                    // consecutive, is one bulk copy announced to the barrier just before it
                    // is issued; absent cells are zeroed.  One lane arrives after the warp
                    // has issued everything, so the phase cannot complete early.
                    uint64_t* bar = &s_bar[(gstep + s) % NST];
                    if (ltid < EY) {
                        asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
                        const int64_t row = (int64_t)pr1[ltid] + r2;
                        const int64_t wbase = (int64_t)b * G.RW + row * G.W;
                        T* dst = st + ltid * SROW;
                        for (int k = 0; k < s_nrun; k++) {
                            const int u0 = s_run[k][0], x0 = s_run[k][1], len = s_run[k][2];
                            const int w0 = x0 >> 6, sh = x0 & 63;
                            const bool two = sh + len > 64;  // the run reaches into word w0+1
                            const uint64_t ua = P.in.ubits[wbase + w0];
                            const uint64_t ub = two ? P.in.ubits[wbase + w0 + 1] : 0ull;
                            const uint32_t oa = P.in.woff[wbase + w0];
                            const uint32_t ob = two ? P.in.woff[wbase + w0 + 1] : 0u;
                            const uint64_t lenmask = (1ull << len) - 1ull;  // len <= EX < 64
                            // bit u: cell x0 + u holds the block (sh >= 43 whenever two)
                            uint64_t pm = (P.in.kbits[wbase + w0] & ua) >> sh;
                            if (two) pm |= (P.in.kbits[wbase + w0 + 1] & ub) << (64 - sh);
                            pm &= lenmask;
                            uint64_t absent = ~pm & lenmask;
                            while (absent) {
                                const int u = __ffsll((long long)absent) - 1;
                                absent &= absent - 1ull;
                                float4* z = reinterpret_cast<float4*>(dst + (u0 + u) * NV);
                                const float4 zero = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
                                for (int k2 = 0; k2 < PC; k2++) z[k2] = zero;
                            }
                            uint64_t m = pm;
                            while (m) {
                                const int u = __ffsll((long long)m) - 1;
                                const int rl = __ffsll((long long)~(m >> u)) - 1;  // run length
                                const int x = x0 + u;
                                const bool lo = (x >> 6) == w0;
                                const int64_t r = (int64_t)(lo ? oa : ob) +
                                                  __popcll((lo ? ua : ub) & ((1ull << (x & 63)) - 1ull));
                                const unsigned bytes = (unsigned)(rl * NV * sizeof(T));
                                mbar_add_tx(bar, bytes);
                                bulk_g2s(dst + (u0 + u) * NV, ipool + ibase + r * NV, bytes, bar);
                                m &= ~(((1ull << rl) - 1ull) << u);
                            }
                        }
                    }
                    __syncwarp();
                    if (ltid == 0) mbar_arrive(bar);
                } else {
                    for (int k = ltid; k < EX * EY * PC; k += NLD) {
                        int cell = k / PC, piece = k - cell * PC;
                        int u1 = cell / EX, u0 = cell - u1 * EX;
                        int x = px0[u0] + px1[u1] + x2;
                        int64_t row = (int64_t)pr0[u0] + pr1[u1] + r2;
                        int64_t r = dense_in ? row * G.n[0] + x : cell_rank(P.in, G, b, x, row, true);
                        constexpr int PE = 16 / (int)sizeof(T);  // values per piece
                        const T* src = r >= 0 ? ipool + ibase + r * NV + PE * piece : ipool;
                        cp_async16(st + u1 * SROW + u0 * NV + PE * piece, src, r >= 0 ? 16 : 0);
                    }
                }
                if constexpr (kCodec != 0) {
                    // chunk scales of the staged cells, one 4-byte copy each (0 for an absent
                    // cell, whose codes are zero), in this plane's cp.async group
                    float* sc = isc + (s % NST) * EY * EX;
                    for (int c = ltid; c < EX * EY; c += NLD) {
                        const int u1 = c / EX, u0 = c - u1 * EX;
                        const int x = px0[u0] + px1[u1] + x2;
                        const int64_t row = (int64_t)pr0[u0] + pr1[u1] + r2;
                        const int64_t r = dense_in ? row * G.n[0] + x : cell_rank(P.in, G, b, x, row, true);
                        cp_async4(sc + c, r >= 0 ? P.in.scale + ibase / NV + r : P.in.scale, r >= 0 ? 4 : 0);
                    }
                }
            }
            cp_async_commit();
        };
        auto wait_plane = [&](int s) {
            if (bulk || sbulk) {
                uint64_t* bar = &s_bar[(gstep + s) % NST];
                const unsigned parity = ((gstep + s) / NST) & 1u;
                if (P.report_late && !mbar_test_wait(bar, parity)) atomicOr(&P.ctr->error, 4);
                unsigned polls = 0;
                const uint64_t t0 = globaltimer_ns();
                while (!mbar_try_wait(bar, parity)) {
                    if (++polls > kMaxPolls || ((polls & 63u) == 0 && globaltimer_ns() - t0 > kWaitNs)) {
                        atomicOr(&P.ctr->error, 4);
                        s_abort[s & 1] = 1;  // the CTA stops after this plane's barrier
                        break;
                    }
                }
            } else if (loader) {
                cp_async_wait<NST - 2>();
            }
        };
        auto out_ranks = [&](int s) {  // sparse output slots of the plane completed at s
            const int zo = out_of(s);
            if (dense_out || s < FIRST || zo < 0 || zo >= n2) return;
            int* orow = orank + (s & 3) * TX * TY;
            if (a0 == 0) {
                // one tile row per lane of the second loader warp: its TX cells lie in one
                // bitmap word (t0 is a multiple of TX, which divides 64)
                const int j = ltid - 32;
                if (j >= 0 && j < TY) {
                    int64_t wbase = -1;
                    if (j < e1) {
                        const int64_t row = (int64_t)rpart(a1, t1 + j, ny) + rpart(a2, zo, ny);
                        wbase = (int64_t)b * G.RW + row * G.W + (t0 >> 6);
                    }
                    const uint64_t uw = wbase >= 0 ? P.out.ubits[wbase] : 0ull;
                    const uint32_t ow = wbase >= 0 ? P.out.woff[wbase] : 0u;
#pragma unroll
                    for (int i = 0; i < TX; i++) {
                        const int bit = (t0 + i) & 63;
                        const bool has = i < e0 && ((uw >> bit) & 1ull);
                        orow[j * TX + i] = has ? (int)(ow + __popcll(uw & ((1ull << bit) - 1ull))) : -1;
                    }
                }
                return;
            }
            for (int c = ltid; c < TX * TY; c += NLD) {
                int j = c / TX, i = c - j * TX;
                int r = -1;
                if (i < e0 && j < e1) {
                    int x = xpart(a0, t0 + i) + xpart(a1, t1 + j) + xpart(a2, zo);
                    int64_t row = (int64_t)rpart(a0, t0 + i, ny) + rpart(a1, t1 + j, ny) + rpart(a2, zo, ny);
                    r = (int)cell_rank(P.out, G, b, x, row, false);
                }
                orow[c] = r;
            }
        };
        auto keep_flags = [&](int s) {  // per-chunk keep flags of the plane completed at s
            const int zo = out_of(s);
            if (s < FIRST || zo < 0 || zo >= n2) return;
            const unsigned* km = kb + (s % 3) * 16;
            for (int c = ltid; c < TX * TY; c += NLD) {
                int j = c / TX, i = c - j * TX;
                if (i >= e0 || j >= e1) continue;
                int64_t r;
                if (dense_out) {
                    int x = xpart(a0, t0 + i) + xpart(a1, t1 + j) + xpart(a2, zo);
                    int64_t row = (int64_t)rpart(a0, t0 + i, ny) + rpart(a1, t1 + j, ny) + rpart(a2, zo, ny);
                    r = row * G.n[0] + x;
                } else {
                    r = orank[(s & 3) * TX * TY + c];
                }
                if (r < 0) continue;
                int hh = j / L, jj = j - hh * L;
                if ((km[hh * 8 + (i >> 1)] >> (16 * (i & 1) + jj)) & 1u) P.keepq[(okeep + r) * 4 + q] = 1;
            }
        };

        const bool cvalid = ci < e0;
        // streamed windows: with one walking direction per item, rows (2i, 2i+1) share a
        // packed pair (their velocity cell, hence their constants, is the same)
        static_assert(L % 2 == 0, "packed streamed windows pair the rows of a segment");
        Walk2<kLim> zu[kZUni ? L / 2 : 1];
        Slide<kLim> zg[kZUni ? 1 : L];
        const WalkConst2 kz = pack_const(kw[2], kw[2]);
#pragma unroll
        for (int j = 0; j < (kZUni ? L / 2 : 1); j++) zu[j].reset();
#pragma unroll
        for (int j = 0; j < (kZUni ? 1 : L); j++) zg[j].reset();
        float msum = 0.0f, mcomp = 0.0f;  // Kahan-compensated FP32 mass of this thread

        if (loader) {
            issue_plane(0);
            issue_plane(1);
        }
        // 16-bit storage with bulk-staged planes: the scales of a plane come by cp.async,
        // which the staging barrier does not cover.  Plane 0's are waited for here; from
        // then on the loaders wait for plane s+1's in step s, before its second barrier.
        if (kCodec != 0 && (bulk || sbulk)) {
            if (loader) cp_async_wait<NST - 2>();
            __syncthreads();
        }

        // one streamed plane; kEmit: the plane completes an output plane
        auto step = [&](int s, auto emit_tag) -> bool {
            constexpr bool kEmit = decltype(emit_tag)::value;
            wait_plane(s);
            // Bulk-staged planes: each thread's barrier wait makes plane s visible to it,
            // and every buffer written in this half of the step is one that no thread
            // can still be reading from the previous step: xbuf is double-buffered, the
            // output ranks have four slots, the keep-flag words three, the flags are
            // taken two planes late, and the stage refilled now was last read before the
            // previous step's second barrier.  cp.async-staged planes need the barrier.
            if (!(bulk || sbulk)) __syncthreads();
            if (!loader) {
                // sweep 0 along axis 0 on halo row `hi`
                const T* line = stage + (s % NST) * S::STAGE + hi * SROW + v;
                const float* lsc = isc + (s % NST) * EY * EX + hi * EX;  // 16-bit: chunk scales
                float* xo = xbuf + (s & 1) * S::XBUF + hi * XROW + v;
                Walk<kLim> wk;
                wk.reset();
                if (kw[0].up) {
#pragma unroll
                    for (int t = 0; t < TX + 5; t++) {
                        float r = wk.push(C::dec(line[t * NV], kCodec ? lsc[t] : 1.0f), kx);
                        if (t >= 5) xo[(t - 5) * NV] = r;
                    }
                } else {
#pragma unroll
                    for (int t = 0; t < TX + 5; t++) {
                        float r = wk.push(C::dec(line[(TX + 5 - t) * NV], kCodec ? lsc[TX + 5 - t] : 1.0f), kx);
                        if (t >= 5) xo[(TX + 4 - t) * NV] = r;
                    }
                }
            } else {
                keep_flags(s - 2);
                out_ranks(s + 1);
                issue_plane(s + NST - 1);
                if (kCodec != 0 && (bulk || sbulk)) cp_async_wait<NST - 2>();  // plane s+1's scales
            }
            __syncthreads();  // sweep-0 rows complete
            // a staging wait of this plane ran out: no sweep on an incomplete plane.  The
            // flag is per plane parity, so no thread's wait on plane s+1 can change what
            // the others read here.
            if (s_abort[s & 1]) return true;
            // sweep 1 along axis 1 over rows j0..j0+L-1 of tile column ci, each output
            // pushed straight into the streamed window of its cell (sweep 2)
            const int zo = out_of(s);
            T* dst = opool + obase + v +
                         ((int64_t)(t0 + ci) * P.stride[a0] + (int64_t)(t1 + j0) * P.stride[a1] +
                          (int64_t)zo * P.stride[a2]) * NV;
            const int64_t dstep = P.stride[a1] * NV;
            const bool fast = dense_out && full;
            const int* orow = orank + (s & 3) * TX * TY + j0 * TX + ci;
            float psum = 0.0f;
            unsigned kmask = 0;
            // new value of row jj.  16-bit storage: the 16 lanes of a half warp hold the 16
            // values of one chunk of one cell, and lane groups that walk sweep 1 in
            // opposite directions (a block straddling v = 0 along axis 1) produce the
            // rows in opposite orders, so the rows are collected first and stored after
            // the walk, by every lane together
            auto store_row = [&](int jj, float res) {
                if (kEmit) {
                    T code;
                    float sco = 1.0f;  // 16-bit storage: the chunk's new scale
                    if constexpr (kCodec != 0) {
                        const ChunkScale cs = chunk_scale(group_max<16>(fabsf(res)));
                        code = C::enc(res, cs.inv);
                        res = C::dec(code, cs.s);  // the value the state now holds
                        sco = cs.s;
                    } else {
                        code = res;
                    }
                    if (fast) {
                        dst[jj * dstep] = code;
                        if (kCodec != 0 && v == 0) P.out.scale[((dst - opool) + jj * dstep) >> 4] = sco;
                        psum += res;
                    } else {
                        int64_t r = -1;
                        if (dense_out) {
                            if (cvalid && j0 + jj < e1) r = 0;
                        } else {
                            r = orow[jj * TX];
                        }
                        if (r >= 0) {
                            int64_t e;  // element offset of the value in the output pool
                            if (dense_out) e = (dst - opool) + jj * dstep;
                            else e = obase + r * NV + v;
                            opool[e] = code;
                            if (kCodec != 0 && v == 0) P.out.scale[e >> 4] = sco;
                            psum += res;
                        }
                    }
                    if (res >= P.thr) kmask |= 1u << jj;
                }
            };
            float rows[kCodec ? L : 1];
            auto emit = [&](int jj, float res) {
                if constexpr (kCodec != 0) rows[jj] = res;
                else store_row(jj, res);
            };
            // sweep-1 output of row jj into its streamed window; rows are produced in
            // walking order (ascending when kUp), and a packed pair is pushed once both
            // of its rows are in, then emitted in that same order
            float pend = 0.0f;
            auto consume = [&](int jj, float yv, auto up_tag) {
                constexpr bool kUp = decltype(up_tag)::value;
                if constexpr (kZUni) {
                    if ((jj & 1) == (kUp ? 0 : 1)) {
                        pend = yv;  // first row of its pair
                        return;
                    }
                    const int lo = kUp ? jj - 1 : jj;
                    const float2 r = zu[lo >> 1].push(kUp ? make_float2(pend, yv) : make_float2(yv, pend), kz);
                    if (kUp) {
                        emit(lo, r.x);
                        emit(lo + 1, r.y);
                    } else {
                        emit(lo + 1, r.y);
                        emit(lo, r.x);
                    }
                } else {
                    emit(jj, zg[jj].push(yv, ks2));
                }
            };
            const float* line = xbuf + (s & 1) * S::XBUF + (j0 * XROW) + ci * NV + v;
            Walk<kLim> wk;
            wk.reset();
            if (kw[1].up) {
#pragma unroll
                for (int t = 0; t < L + 5; t++) {
                    float r = wk.push(line[t * XROW], kw[1]);
                    if (t >= 5) consume(t - 5, r, std::true_type{});
                }
            } else {
#pragma unroll
                for (int t = 0; t < L + 5; t++) {
                    float r = wk.push(line[(L + 5 - t) * XROW], kw[1]);
                    if (t >= 5) consume(L + 4 - t, r, std::false_type{});
                }
            }
            if constexpr (kCodec != 0) {
#pragma unroll
                for (int jj = 0; jj < L; jj++) store_row(jj, rows[jj]);
            }
            if (kEmit) {
                unsigned km = __reduce_or_sync(0xffffffffu, kmask << (16 * (ci & 1)));
                if (lane == 0) kb[(s % 3) * 16 + warp] = km;
                float y = psum - mcomp;
                float t = msum + y;
                mcomp = (t - msum) - y;
                msum = t;
            }
            return false;
        };
        int s = 0;
        bool stop = false;
        for (; s < FIRST && !stop; s++) stop = step(s, std::false_type{});
        for (; s < nsteps && !stop; s++) stop = step(s, std::true_type{});
        if (stop) {
            s--;  // the plane whose wait ran out
            // leave no copy in flight: plane s ran out, planes s+1 .. s+NST-1 may have been
            // issued; wait (bounded) for each before the CTA exits
            if (bulk || sbulk) {
                if (ltid == 0)
                    for (int p = s; p < min(s + NST, nsteps); p++) {
                        uint64_t* bar = &s_bar[(gstep + p) % NST];
                        const unsigned parity = ((gstep + p) / NST) & 1u;
                        unsigned polls = 0;
                        const uint64_t t0 = globaltimer_ns();
                        while (!mbar_try_wait(bar, parity) && ++polls <= kMaxPolls &&
                               ((polls & 63u) != 0 || globaltimer_ns() - t0 <= kWaitNs)) {
                        }
                    }
            } else {
                cp_async_wait<0>();
            }
            break;
        }

        __syncthreads();
        if (loader) {
            keep_flags(nsteps - 2);
            keep_flags(nsteps - 1);
        }
        cp_async_wait<0>();
        if (bulk || sbulk) gstep += (unsigned)nsteps;
        double m = (double)msum;
        for (int o = 16; o > 0; o >>= 1) m += __shfl_xor_sync(0xffffffffu, m, o);
        if (lane == 0 && m != 0.0) atomicAdd(&P.ctr->mass, m);
    }
    if (P.cta_done && tid == 0) P.cta_done[blockIdx.x] = globaltimer_ns();
}

// ---- work list ------------------------------------------------------------------
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
    if (aborted(G.abort)) return;
    int64_t ntiles = (int64_t)T.ntile0 * T.ntile1;
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (int64_t)G.nb * ntiles) return;
    int b = (int)(i / ntiles);
    int tile = (int)(i - (int64_t)b * ntiles);
    int lo[3], hi[3];
    lo[T.ax[0]] = (tile % T.ntile0) * TX;
    hi[T.ax[0]] = min(lo[T.ax[0]] + TX, G.n[T.ax[0]]);
    lo[T.ax[1]] = (tile / T.ntile0) * T.ty;
    hi[T.ax[1]] = min(lo[T.ax[1]] + T.ty, G.n[T.ax[1]]);
    lo[T.ax[2]] = 0;
    hi[T.ax[2]] = G.n[T.ax[2]];
    const uint64_t* seg = T.ubits + (int64_t)b * G.RW;
    bool any = false;
    for (int z = lo[2]; z < hi[2] && !any; z++)
        for (int y = lo[1]; y < hi[1] && !any; y++)
            any = row_any(seg + ((int64_t)y + (int64_t)G.n[1] * z) * G.W, lo[0], hi[0]);
    flags[i] = any ? 1u : 0u;
}

// flat: the item is the pair's index b * ntiles + tile itself (the caller needs no
// search of item_base to find b)
__global__ void k_tile_items(int64_t ntiles, int nb, const uint32_t* __restrict__ flags,
                             const uint32_t* __restrict__ pos, const int64_t* __restrict__ base,
                             uint32_t* __restrict__ items, int flat, const int* abort)
{
    if (aborted(abort)) return;
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (int64_t)nb * ntiles) return;
    if (!flags[i]) return;
    int b = (int)(i / ntiles);
    items[base[b] + pos[i]] = (uint32_t)(flat ? i : i - (int64_t)b * ntiles);
}

inline int nblk(int64_t n, int t) { return (int)((n + t - 1) / t); }

template <int TY, bool kLim, bool kZUni, int kCodec = 0, bool kRed = false>
vl_status launch_fused(Grid* g, const FusedArgs& P)
{
    auto kern = k_fused<TY, kLim, kZUni, kCodec, kRed>;
    const int smem = Shape<TY, (int)sizeof(typename Codec<kCodec>::T)>::SMEM;
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    int nsm = 0, per_sm = 0;
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, g->dev.device);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, NT, smem);
    if (per_sm < 1) per_sm = 1;
    FusedArgs Q = P;
    const int nct = nsm * per_sm;
    if (nct > kMaxCtas) Q.cta_done = nullptr;
    g->cta_count = Q.cta_done ? nct : 0;
    g->cta_groups = 1;
    kern<<<nct, NT, smem, g->stream>>>(Q);
    note_launch();
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(g, e, "fused sweep launch");
    return VL_OK;
}

}  // namespace

// Compaction of g->tile_flags ([nb][ntiles] 0/1) into the work list: items[item_base[b]
// .. item_base[b+1]) = the flagged tiles of block id b in ascending order (flat: as
// b * ntiles + tile).
void launch_items_from_flags(Grid* g, int64_t ntiles, bool flat)
{
    const GridGeom& G = g->geom;
    const int64_t need = ntiles * G.nb;
    launch_seg_scan(g->tile_flags, g->tile_pos, g->item_cnt, ntiles, G.nb, g->stream, G.abort);
    launch_base_scan(g->item_cnt, g->item_base, G.nb, g->stream, G.abort);
    k_tile_items<<<nblk(need, 256), 256, 0, g->stream>>>(ntiles, G.nb, g->tile_flags, g->tile_pos,
                                                           g->item_base, g->items, flat ? 1 : 0, G.abort);
    note_launch();
}

// Work list of a fused launch: one item per (block id, tile column) holding any slot of
// the next layout, grouped by block id (item_base[b] .. item_base[b+1]).
void launch_tile_list(Grid* g, const TileArgs& T, int64_t need, int64_t ntiles)
{
    k_tile_flags<<<nblk(need, 256), 256, 0, g->stream>>>(T, g->tile_flags);
    note_launch();
    launch_items_from_flags(g, ntiles, false);
}

// Work-list buffers for `need` (block id, tile) pairs (allocated before any captured
// step sequence; they never shrink).
vl_status worklist_reserve(Grid* g, int64_t need)
{
    if (need > 0xffffffffLL) return fail(g, VL_EINVAL, "work list: more than 2^32 (block id, tile) pairs");
    if (need <= g->ntiles_alloc) return VL_OK;
    g->release(g->tile_flags);
    g->release(g->tile_pos);
    g->release(g->items);
    g->tile_flags = (uint32_t*)g->alloc((size_t)need * 4);
    g->tile_pos = (uint32_t*)g->alloc((size_t)need * 4);
    g->items = (uint32_t*)g->alloc((size_t)need * 4);
    if (!g->tile_flags || !g->tile_pos || !g->items) {
        g->ntiles_alloc = 0;
        return fail(g, VL_ENOMEM, "work-list allocation failed");
    }
    g->ntiles_alloc = need;
    return VL_OK;
}

// Work-list buffers of the fused form for this sweep order (allocated before any
// captured step sequence).
// Tile rows along the second sweep axis: 16 when the streamed axis is the velocity
// chunk's own axis (unless 8 is asked for), 8 otherwise.
int tile_rows(const StepArgs& a) { return (a.order[2] == 2 && a.tile[1] != 8) ? 16 : 8; }

vl_status fused_worklist_alloc(Grid* g, const StepArgs& a)
{
    const GridGeom& G = g->geom;
    const int ty = tile_rows(a);
    const int64_t ntiles = (int64_t)((G.n[a.order[0]] + TX - 1) / TX) * ((G.n[a.order[1]] + ty - 1) / ty);
    return worklist_reserve(g, ntiles * G.nb);
}

vl_status run_fused(Grid* g, const StepArgs& a)
{
    if (use_gt3(g, a)) return run_gt3(g, a);
    const GridGeom& G = g->geom;
    Layout& A = g->lay[g->cur];
    Layout& B = g->lay[1 - g->cur];
    int ax[3] = {a.order[0], a.order[1], a.order[2]};
    const bool zuni = ax[2] == 2;  // the streamed axis is the chunk's (vz) axis
    const int ty = tile_rows(a);
    int ntile0 = (G.n[ax[0]] + TX - 1) / TX;
    int ntile1 = (G.n[ax[1]] + ty - 1) / ty;
    int64_t ntiles = (int64_t)ntile0 * ntile1;
    if (ntiles > 0xffffffffLL) return fail(g, VL_EINVAL, "fused form: too many tiles");
    int64_t need = ntiles * G.nb;
    vl_status wst = fused_worklist_alloc(g, a);
    if (wst != VL_OK) return wst;
    TileArgs T;
    T.G = G;
    T.ubits = B.ubits;
    for (int j = 0; j < 3; j++) T.ax[j] = ax[j];
    T.ntile0 = ntile0;
    T.ntile1 = ntile1;
    T.ty = ty;
    launch_tile_list(g, T, need, ntiles);

    FusedArgs P;
    P.G = G;
    P.in = A.view();
    P.out = B.view();
    P.stride[0] = 1;
    P.stride[1] = G.n[0];
    P.stride[2] = (int64_t)G.n[0] * G.n[1];
    for (int j = 0; j < 3; j++) P.ax[j] = ax[j];
    P.walk = a.walk;
    P.sweep = a.sweep;
    P.nvmax = a.nvmax;
    P.thr = (float)g->threshold;
    P.ntile0 = ntile0;
    P.items = g->items;
    P.item_base = g->item_base;
    P.keepq = B.keepq;
    P.ctr = a.ctr;
    P.report_late = fault_requested("timeout") ? 1 : 0;
    P.cta_done = a.stamp_ctas ? g->cta_done : nullptr;
    P.gt_k = a.ghost;
    record_sweep_event(a.ev0, g->stream, a.ev_node);
    vl_status st = VL_OK;
    if (a.ghost != 3) {
        // reduced ghost depth: compiled for FP32 storage only (the host checks)
        if (zuni && ty == 16)
            st = a.limiter ? launch_fused<16, true, true, 0, true>(g, P) : launch_fused<16, false, true, 0, true>(g, P);
        else if (zuni)
            st = a.limiter ? launch_fused<8, true, true, 0, true>(g, P) : launch_fused<8, false, true, 0, true>(g, P);
        else
            st = a.limiter ? launch_fused<8, true, false, 0, true>(g, P) : launch_fused<8, false, false, 0, true>(g, P);
    } else {
        with_codec(g->codec, [&](auto c) {
            constexpr int kc = decltype(c)::value;
            if (zuni && ty == 16)
                st = a.limiter ? launch_fused<16, true, true, kc>(g, P) : launch_fused<16, false, true, kc>(g, P);
            else if (zuni)
                st = a.limiter ? launch_fused<8, true, true, kc>(g, P) : launch_fused<8, false, true, kc>(g, P);
            else
                st = a.limiter ? launch_fused<8, true, false, kc>(g, P) : launch_fused<8, false, false, kc>(g, P);
        });
    }
    record_sweep_event(a.ev1, g->stream, a.ev_node);
    return st;
}

// Launch of the fused kernel over caller-provided buffers of a dense layout (every
// cell holds every block id): `in`/`out` carry cnt/base/dense arrays and pools, items and
// item_base list every (block id, tile) pair, ctab holds the constant tables.  Used by the
// allocation-free entry point; the step's sparsity rule is not applied (threshold +inf).
vl_status launch_fused_dense(const GridGeom& G, const LayoutView& in, const LayoutView& out,
                             const int order[3], int limiter, const float4* ctab, int nvmax,
                             const uint32_t* items, const int64_t* item_base, int ntile0,
                             StepCounters* ctr, int device, cudaStream_t stream)
{
    FusedArgs P;
    P.G = G;
    P.in = in;
    P.out = out;
    P.stride[0] = 1;
    P.stride[1] = G.n[0];
    P.stride[2] = (int64_t)G.n[0] * G.n[1];
    for (int j = 0; j < 3; j++) P.ax[j] = order[j];
    P.walk = ctab;
    P.sweep = ctab + 3 * nvmax;
    P.nvmax = nvmax;
    P.thr = INFINITY;
    P.ntile0 = ntile0;
    P.items = items;
    P.item_base = item_base;
    P.keepq = nullptr;
    P.ctr = ctr;
    P.report_late = 0;
    P.cta_done = nullptr;
    P.gt_k = 3;
    Grid tmp;  // launch helper needs the device and the stream only
    tmp.dev.device = device;
    tmp.stream = stream;
    const bool zuni = order[2] == 2;
    if (zuni) return limiter ? launch_fused<16, true, true>(&tmp, P) : launch_fused<16, false, true>(&tmp, P);
    return limiter ? launch_fused<8, true, false>(&tmp, P) : launch_fused<8, false, false>(&tmp, P);
}

int fused_tile_rows(const int order[3]) { return order[2] == 2 ? 16 : 8; }

}  // namespace vlgt
