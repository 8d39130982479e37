// gt3.cu -- Ghost Translation (GT3) on one GPU, plane-batched kernel (paper Section 3).
//
// Same computation as the row-segment kernel of fused.cu: a work item is (block id b,
// velocity chunk q, tile of 16 x 16 cells across the two in-plane axes); the tile plus
// its 3-cell ghost halo (Section 3.1: the 2-cell stencil and one face neighbour) is
// staged into shared memory plane by plane along the third (streamed) axis, exactly once
// per step, and all three sweeps run on it.  What differs is how the work is laid out on
// the SM:
//   * planes are processed in batches of three.  While the CTA sweeps batch k, the four
//     warps that sit out sweep 1 stage batch k+1, one halo row per thread, with TMA bulk
//     copies (one per contiguous run of a row; 16-byte cp.async for the short run where a
//     dense row wraps around the periodic grid).  The CTA synchronises once per batch
//     after sweep 0; after sweep 1 the sweep-1 warps only arrive on a named barrier that
//     the staging warps wait on, and go on to sweep 2 among themselves;
//   * every walk moves two velocity cells in packed f32x2 registers: sweep 0 runs on the
//     21 halo lines that sweep 1 reads (3 planes x 21 lines x 8 lane pairs = 504 walks),
//     sweep 1 on the 16 tile lines (384 walks), both in place in shared memory;
//   * sweep 2 is streamed: each compute thread keeps the windows of four velocity cells
//     (one vx row of a chunk) of two tile cells in registers, reads them with 16-byte
//     shared loads and writes 16-byte global stores, so a warp writes 8 whole cells.
// All walks start on the upwind side (Walk2), so the velocity cells of an item must all
// move the same way along each axis: no velocity block may straddle v_d = 0 (the host
// checks), and the streamed axis must not be x (the chunk's vx cells have different
// Courant numbers along x, and x is the contiguous axis of the staged rows).
#include <cuda_runtime.h>
#include <stdint.h>

#include <cmath>

#include "grid.h"

namespace vlgt {

namespace {

constexpr int kT = 16;                      // tile edge along both in-plane axes
constexpr int kE = kT + 2 * kHalo;          // 22 staged cells per in-plane axis
constexpr int kRP = kE * kChunk + 16;       // staged row pitch in floats: rows 16 banks apart
constexpr int kPS = kE * kRP + 16;          // plane pitch in floats
constexpr int kNB = 3;                      // planes per batch
constexpr int kNC = 512;                    // threads (16 warps)
constexpr int kNT = kNC;
constexpr int kLines = kT + 5;              // sweep-0 lines: those sweep 1 reads
constexpr int kNX = kNB * kLines * 8;       // sweep-0 walks per batch (lane pairs)
constexpr int kNY = kNB * kT * 8;           // sweep-1 walks per batch
constexpr int kNS = kNC - kNY;              // staging threads: those that sit out sweep 1
constexpr int kFirst = kHalo + 2;           // first streamed plane that completes an output
// 16-bit storage with sweep 0 along x: the codes of a staged row are packed (8 floats per
// cell) at the end of the row that sweep 0 reaches last -- from float kCodesHi when it
// walks up, from float 0 when it walks down
constexpr int kCodesHi = kRP - kE * kChunk / 2;
static_assert(kNX <= kNC && kNY <= kNC, "walks of a batch must fit the compute threads");
static_assert(kT * kT * 4 == 2 * kNC, "sweep 2: two tile cells x one vx row per thread");
static_assert(kNS == 128, "staging threads: warps 12-15 (named barrier 1)");

struct Gt3Smem {
    float buf[2][kNB][kPS];   // staged planes, swept in place (two batches in flight)
    int orank[2][kNB][kT * kT];  // sparse output slots of the tile cells, per plane
    float4 kc[3][kChunk];     // WalkConst (g, A, B, up) per sweep and velocity cell
    int run[2][kE][3];        // per item parity: contiguous runs of a staged row along x
    int rrow[2][kE];          // per item parity: row-space part of each staged row
    int xs[2][kE];            // per item parity: x of each staged column
    uint64_t bar[2];          // staging barriers, one per batch buffer
    long long work;           // the current work item
    long long next;           // the one after it (taken while the current one runs)
    int nrun[2];
    int pref;                 // batch 0 of the current item was staged during the last one
    int abort;
};
// 16-bit storage: the chunk scales of the staged cells, [2][kNB][kE][kSP] floats after
// Gt3Smem (per batch buffer and plane, staged row-major like the cells).  The row pitch
// is odd, so that the staging threads, one per row, write 32 different banks.
constexpr int kSP = kE + 1;
constexpr int kScales = 2 * kNB * kE * kSP;
template <int kCodec>
constexpr size_t smem_bytes() { return sizeof(Gt3Smem) + (kCodec ? kScales * sizeof(float) : 0); }
__device__ __forceinline__ float* scales_of(Gt3Smem& S) { return reinterpret_cast<float*>(&S + 1); }
static_assert(smem_bytes<1>() <= 227 * 1024, "shared memory of one CTA");

struct Gt3Args {
    GridGeom G;
    LayoutView in, out;
    int ax[3];          // physical axis of sweep 0, 1, 2 (axis 2 is streamed, never x)
    int ar;             // the in-plane axis that is not x
    int64_t stride[3];  // cell-index stride of each physical axis (1, nx, nx*ny)
    const float4* walk; // [3][nvmax] WalkConst (g, A, B, up) per axis and velocity index
    int nvmax;
    float thr;
    int ntile0;         // tiles along x
    const uint32_t* items;
    const int64_t* item_base;  // [nb + 1]
    uint8_t* keepq;
    StepCounters* ctr;
    int report_late;    // testing hook: a staging wait not complete at its first poll is
                        // reported as overdue (VL_ETIMEOUT), then waited for
    uint64_t* cta_done; // optional [gridDim.x]: %globaltimer when the CTA ran out of work
};

__device__ __forceinline__ unsigned su32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void bar_init(uint64_t* bar, unsigned count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(su32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void bar_add_tx(uint64_t* bar, unsigned bytes)
{
    asm volatile("mbarrier.expect_tx.relaxed.cta.shared::cta.b64 [%0], %1;\n" ::"r"(su32(bar)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void bar_arrive(uint64_t* bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(su32(bar)) : "memory");
}
__device__ __forceinline__ bool bar_try(uint64_t* bar, unsigned parity)
{
    unsigned ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(su32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ bool bar_test(uint64_t* bar, unsigned parity)
{
    unsigned ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(su32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ uint64_t now_ns()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;\n" : "=l"(t));
    return t;
}
__device__ __forceinline__ void copy_g2s(void* dst, const void* src, unsigned bytes, uint64_t* bar)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(
            su32(dst)),
        "l"(src), "r"(bytes), "r"(su32(bar))
        : "memory");
}
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory"); }
// 16-byte copy global -> shared; src_bytes = 0 fills the 16 bytes with zeros
__device__ __forceinline__ void cp16(void* dst, const void* src, int src_bytes)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(su32(dst)), "l"(src), "r"(src_bytes)
                 : "memory");
}
// 4-byte copy global -> shared; src_bytes = 0 writes 0
__device__ __forceinline__ void cp4(void* dst, const void* src, int src_bytes)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(su32(dst)), "l"(src), "r"(src_bytes)
                 : "memory");
}
// the barrier's pending count drops by one once this thread's earlier cp.async copies land
__device__ __forceinline__ void cp_arrive(uint64_t* bar)
{
    asm volatile("cp.async.mbarrier.arrive.noinc.shared::cta.b64 [%0];\n" ::"r"(su32(bar)) : "memory");
}

// Two 16-bit codes (lanes l, l+1) as floats times their chunk's scale, as Codec::dec
// does per value (the scale is a power of two: exact).
template <int kCodec>
__device__ __forceinline__ float2 dec2(uint32_t w, float2 s)
{
    float2 f;
    if constexpr (kCodec == 1) f = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&w));
    else f = __half22float2(*reinterpret_cast<const __half2*>(&w));
    return mul2(f, s);
}
// Two floats times 1/scale rounded to 16-bit codes, as Codec::enc does per value.
template <int kCodec>
__device__ __forceinline__ uint32_t enc2(float2 f, float2 inv)
{
    const float2 x = mul2(f, inv);
    uint32_t w;
    if constexpr (kCodec == 1) {
        const __nv_bfloat162 h = __float22bfloat162_rn(x);
        w = *reinterpret_cast<const uint32_t*>(&h);
    } else {
        const __half2 h = __float22half2_rn(x);
        w = *reinterpret_cast<const uint32_t*>(&h);
    }
    return w;
}

// A staging wait gives up after one second of device time or 2^24 polls (a batch is a
// few tens of kB staged in microseconds): reaching either means a fault upstream.
constexpr unsigned kPolls = 1u << 24;
constexpr uint64_t kWaitLimitNs = 1000000000ull;

__device__ __forceinline__ bool bar_wait_bounded(uint64_t* bar, unsigned parity)
{
    unsigned polls = 0;
    const uint64_t t0 = now_ns();
    while (!bar_try(bar, parity)) {
        if (++polls > kPolls || ((polls & 63u) == 0 && now_ns() - t0 > kWaitLimitNs)) return false;
    }
    return true;
}

__device__ __forceinline__ float2 lds2(const float* p) { return *reinterpret_cast<const float2*>(p); }
__device__ __forceinline__ void sts2(float* p, float2 v) { *reinterpret_cast<float2*>(p) = v; }

// row-space contribution (row = y + ny*z) of coordinate c along physical axis d (1 or 2)
__device__ __forceinline__ int rowpart(int d, int c, int ny) { return d == 1 ? c : c * ny; }

// One work item: block id b, velocity chunk q, tile origin and extent.
struct Item {
    int b, q, tx0, tr0, ex, er;
    bool dense_in, dense_out, up0, up2;
    int64_t ibase, obase;
};

__device__ __forceinline__ Item decode_item(const Gt3Args& P, int64_t w)
{
    const GridGeom& G = P.G;
    int lo = 0, hb = G.nb;  // items are grouped by b, q-major then tile
    while (hb - lo > 1) {
        const int mid = (lo + hb) >> 1;
        if (4 * P.item_base[mid] <= w) lo = mid;
        else hb = mid;
    }
    Item it;
    it.b = lo;
    const int64_t mb = P.item_base[lo + 1] - P.item_base[lo];
    const int64_t wl = w - 4 * P.item_base[lo];
    it.q = (int)(wl / mb);
    const uint32_t tile = P.items[P.item_base[lo] + (wl % mb)];
    it.tx0 = (int)(tile % P.ntile0) * kT;
    it.tr0 = (int)(tile / P.ntile0) * kT;
    it.ex = min(kT, G.n[0] - it.tx0);
    it.er = min(kT, G.n[P.ar] - it.tr0);
    it.dense_in = (P.in.dense[lo] & 3) == 3;
    it.dense_out = (P.out.dense[lo] & 1) != 0;
    it.ibase = ((int64_t)P.in.base[lo] * 4 + (int64_t)it.q * P.in.cnt[lo]) * kChunk;
    it.obase = ((int64_t)P.out.base[lo] * 4 + (int64_t)it.q * P.out.cnt[lo]) * kChunk;
    // direction along the streamed axis (not x: the same for every velocity cell of the
    // item, the host checks that no block straddles v = 0)
    const int d = P.ax[2];
    const int bc = d == 1 ? (lo / G.nbx) % G.nby : lo / (G.nbx * G.nby);
    it.up2 = P.walk[d * P.nvmax + bc * 4 + (d == 2 ? it.q : 0)].w != 0.0f;
    // and along the axis of sweep 0 (uniform for the same reason)
    const int d0 = P.ax[0];
    const int bc0 = d0 == 0 ? lo % G.nbx : (d0 == 1 ? (lo / G.nbx) % G.nby : lo / (G.nbx * G.nby));
    it.up0 = P.walk[d0 * P.nvmax + bc0 * 4 + (d0 == 2 ? it.q : 0)].w != 0.0f;
    return it;
}

// Runs and row parts of an item's staged rows and the x of its staged columns into
// table t (threads kNC-1-2kE .. kNC-1).
__device__ __forceinline__ void item_tables(const Gt3Args& P, Gt3Smem& S, const Item& it, int t, int tid)
{
    const int nx = P.G.n[0], nr = P.G.n[P.ar];
    if (tid >= kNC - 1 - 2 * kE && tid < kNC - 1 - kE) S.xs[t][tid - (kNC - 1 - 2 * kE)] = wrapi(it.tx0 - kHalo + tid - (kNC - 1 - 2 * kE), nx);
    if (tid == kNC - 1) {
        int u0 = 0, nrun = 0;
        while (u0 < kE) {
            const int x = wrapi(it.tx0 - kHalo + u0, nx);
            const int len = min(kE - u0, nx - x);
            S.run[t][nrun][0] = u0;
            S.run[t][nrun][1] = x;
            S.run[t][nrun][2] = len;
            nrun++;
            u0 += len;
        }
        S.nrun[t] = nrun;
    } else if (tid >= kNC - 1 - kE && tid < kNC - 1) {
        const int u = tid - (kNC - 1 - kE);
        S.rrow[t][u] = rowpart(P.ar, wrapi(it.tr0 - kHalo + u, nr), P.G.n[1]);
    }
}

// Staging of batch k of an item (planes kNB k .. kNB k + 2 of its stream) into buffer
// g & 1, g = the CTA's running batch index; run by the kNS staging threads (sl = 0..127),
// one staged row per thread, and every staging thread arrives on the batch's barrier
// once its copies have landed.  Contiguous runs of a row go by TMA bulk copies; the short
// run where a dense row wraps around the periodic grid (kShortRun cells or fewer) goes by
// 16-byte cp.async copies instead: the SM's bulk-copy unit takes a roughly fixed time per
// request, and these runs would add half as many requests again.  The chunk scale of each staged cell goes into the scale table with a 4-byte
// cp.async copy (0 for an absent cell).  With sweep 0 along x the row's codes are packed
// at one end of the row (kCodesHi) by bulk copies per contiguous run: sweep 0 walks
// towards that end and writes its FP32 result two cells behind the one it reads, which
// overwrites only codes read at least three positions earlier.  Otherwise the 32 bytes of
// codes of each cell go to the upper half of its own 64-byte slot with two 16-byte
// cp.async copies, so that each line of sweep 0 overwrites only codes it has read.
constexpr int kShortRun = 4;

// cells of an item's staged row that go by bulk copies (runs longer than kShortRun)
__device__ __forceinline__ int bulk_cells(const Gt3Smem& S, int t)
{
    int c = 0;
    for (int k2 = 0; k2 < S.nrun[t]; k2++)
        if (S.run[t][k2][2] > kShortRun) c += S.run[t][k2][2];
    return c;
}

template <int kCodec, bool kA0X>
__device__ __forceinline__ void stage_batch(const Gt3Args& P, Gt3Smem& S, const Item& it, int t, int k,
                                            unsigned g, int sl)
{
    const GridGeom& G = P.G;
    const int nx = G.n[0], ny = G.n[1], a2 = P.ax[2], n2 = G.n[a2];
    const int nsteps = n2 + kFirst;
    const unsigned slot = g & 1u;
    uint64_t* bar = &S.bar[slot];
    const int nj = min(kNB, nsteps - kNB * k);
    const int nrun = S.nrun[t];
    // staged row (and output row) of this thread: rows go round-robin over the four
    // staging warps, whose lanes issue their copies one after another
    const int sw = (sl & 31) * (kNS / 32) + (sl >> 5);
    const float* ipool = static_cast<const float*>(P.in.pool);
    auto plane_of = [&](int s) { return it.up2 ? s - kHalo : n2 + 2 - s; };
    auto out_of = [&](int s) { return it.up2 ? s - kFirst : n2 + 4 - s; };
    if constexpr (kCodec != 0) {
        using T = typename Codec<kCodec>::T;
        const T* cpool = static_cast<const T*>(P.in.pool) + it.ibase;  // codes of rank 0
        const float* spool = P.in.scale + it.ibase / kChunk;            // scale of rank 0
        if (sw < nj * kE) {
            const int j = sw / kE, rho = sw - j * kE;
            const int pz = wrapi(plane_of(kNB * k + j), n2);
            const int64_t row = (int64_t)S.rrow[t][rho] + rowpart(a2, pz, ny);
            float* drow = &S.buf[slot][j][rho * kRP];
            float* srow = scales_of(S) + ((slot * kNB + j) * kE + rho) * kSP;
            if constexpr (kA0X) {
                float* codes = drow + (it.up0 ? kCodesHi : 0);
                fence_async_smem();
                if (it.dense_in) {
                    const int64_t r0 = row * nx;
                    for (int k2 = 0; k2 < nrun; k2++) {
                        const int u0 = S.run[t][k2][0], x0 = S.run[t][k2][1], len = S.run[t][k2][2];
                        float* d = codes + u0 * (kChunk / 2);
                        const T* src = cpool + (r0 + x0) * kChunk;
                        if (len > kShortRun) {
                            copy_g2s(d, src, (unsigned)(len * kChunk * sizeof(T)), bar);
                        } else {
                            for (int i = 0; i < len * 2; i++) cp16(d + 4 * i, src + 8 * i, 16);
                        }
                    }
                    for (int u = 0; u < kE; u++) cp4(srow + u, spool + r0 + S.xs[t][u], 4);
                } else {
                    // runs of present cells (consecutive slots) as bulk copies, each announced
                    // to the barrier before it is issued; absent cells get zero codes and scale
                    const int64_t wbase = (int64_t)it.b * G.RW + row * G.W;
                    for (int k2 = 0; k2 < nrun; k2++) {
                        const int u0 = S.run[t][k2][0], x0 = S.run[t][k2][1], len = S.run[t][k2][2];
                        const int w0 = x0 >> 6, sh = x0 & 63;
                        const bool two = sh + len > 64;
                        const uint64_t ua = P.in.ubits[wbase + w0];
                        const uint64_t ub = two ? P.in.ubits[wbase + w0 + 1] : 0ull;
                        const uint32_t oa = P.in.woff[wbase + w0];
                        const uint32_t ob = two ? P.in.woff[wbase + w0 + 1] : 0u;
                        const uint64_t lenmask = (1ull << len) - 1ull;  // len <= 22
                        uint64_t pm = (P.in.kbits[wbase + w0] & ua) >> sh;
                        if (two) pm |= (P.in.kbits[wbase + w0 + 1] & ub) << (64 - sh);
                        pm &= lenmask;
                        uint64_t absent = ~pm & lenmask;
                        while (absent) {
                            const int u = u0 + __ffsll((long long)absent) - 1;
                            absent &= absent - 1ull;
                            cp16(codes + u * (kChunk / 2), cpool, 0);
                            cp16(codes + u * (kChunk / 2) + 4, cpool, 0);
                            cp4(srow + u, spool, 0);
                        }
                        uint64_t m = pm;
                        while (m) {
                            const int u = __ffsll((long long)m) - 1;
                            const int rl = __ffsll((long long)~(m >> u)) - 1;
                            const int x = x0 + u;
                            const bool lw = (x >> 6) == w0;
                            const int64_t r = (int64_t)(lw ? oa : ob) + __popcll((lw ? ua : ub) & ((1ull << (x & 63)) - 1ull));
                            const unsigned bytes = (unsigned)(rl * kChunk * sizeof(T));
                            bar_add_tx(bar, bytes);
                            copy_g2s(codes + (u0 + u) * (kChunk / 2), cpool + r * kChunk, bytes, bar);
                            for (int i = 0; i < rl; i++) cp4(srow + u0 + u + i, spool + r + i, 4);
                            m &= ~(((1ull << rl) - 1ull) << u);
                        }
                    }
                }
            } else {
                for (int u = 0; u < kE; u++) {
                    const int x = S.xs[t][u];
                    int64_t r;
                    if (it.dense_in) {
                        r = row * nx + x;
                    } else {
                        const int64_t wi = (int64_t)it.b * G.RW + row * G.W + (x >> 6);
                        const uint64_t bit = 1ull << (x & 63);
                        const uint64_t uw = P.in.ubits[wi];
                        r = ((uw & P.in.kbits[wi] & bit) != 0ull) ? (int64_t)P.in.woff[wi] + __popcll(uw & (bit - 1ull))
                                                                   : -1;
                    }
                    float* dst = drow + u * kChunk + 8;
                    const T* src = r >= 0 ? cpool + r * kChunk : cpool;
                    const int nbytes = r >= 0 ? 16 : 0;
                    cp16(dst, src, nbytes);
                    cp16(dst + 4, src + 8, nbytes);
                    cp4(srow + u, r >= 0 ? spool + r : spool, r >= 0 ? 4 : 0);
                }
            }
        }
        // dense rows with sweep 0 along x: the batch's code bytes, announced without an
        // arrival (the phase also waits for every staging thread's arrival below)
        if (kA0X && it.dense_in && sl == 0)
            bar_add_tx(bar, (unsigned)(nj * kE * bulk_cells(S, t) * kChunk * sizeof(T)));
        cp_arrive(bar);
    } else if (it.dense_in) {
        // the batch's bulk-copy bytes, announced once (the copies of the other staging
        // threads may complete before or after it; the phase also waits for every staging
        // thread's arrival)
        if (sl == 0) bar_add_tx(bar, (unsigned)(nj * kE * bulk_cells(S, t) * kChunk * sizeof(float)));
        if (sw < nj * kE) {
            const int j = sw / kE, rho = sw - j * kE;
            const int pz = wrapi(plane_of(kNB * k + j), n2);
            const int64_t row = (int64_t)S.rrow[t][rho] + rowpart(a2, pz, ny);
            const float* src = ipool + it.ibase + row * nx * kChunk;
            float* dst = &S.buf[slot][j][rho * kRP];
            fence_async_smem();
            for (int k2 = 0; k2 < nrun; k2++) {
                const int u0 = S.run[t][k2][0], x0 = S.run[t][k2][1], len = S.run[t][k2][2];
                if (len > kShortRun) {
                    copy_g2s(dst + u0 * kChunk, src + x0 * kChunk, (unsigned)(len * kChunk * sizeof(float)), bar);
                } else {
                    for (int i = 0; i < len * (kChunk / 4); i++)
                        cp16(dst + u0 * kChunk + 4 * i, src + x0 * kChunk + 4 * i, 16);
                }
            }
        }
        cp_arrive(bar);
    } else {
        // runs of present cells (consecutive slots) as bulk copies, each announced to the
        // barrier before it is issued; absent cells are zeroed.  Each staging thread
        // arrives after announcing its bytes, so the phase cannot end before every
        // announcement.
        if (sw < nj * kE) {
            const int j = sw / kE, rho = sw - j * kE;
            const int pz = wrapi(plane_of(kNB * k + j), n2);
            const int64_t row = (int64_t)S.rrow[t][rho] + rowpart(a2, pz, ny);
            const int64_t wbase = (int64_t)it.b * G.RW + row * G.W;
            float* dst = &S.buf[slot][j][rho * kRP];
            fence_async_smem();
            for (int k2 = 0; k2 < nrun; k2++) {
                const int u0 = S.run[t][k2][0], x0 = S.run[t][k2][1], len = S.run[t][k2][2];
                const int w0 = x0 >> 6, sh = x0 & 63;
                const bool two = sh + len > 64;
                const uint64_t ua = P.in.ubits[wbase + w0];
                const uint64_t ub = two ? P.in.ubits[wbase + w0 + 1] : 0ull;
                const uint32_t oa = P.in.woff[wbase + w0];
                const uint32_t ob = two ? P.in.woff[wbase + w0 + 1] : 0u;
                const uint64_t lenmask = (1ull << len) - 1ull;  // len <= 22
                uint64_t pm = (P.in.kbits[wbase + w0] & ua) >> sh;
                if (two) pm |= (P.in.kbits[wbase + w0 + 1] & ub) << (64 - sh);
                pm &= lenmask;
                uint64_t absent = ~pm & lenmask;
                while (absent) {
                    const int u = __ffsll((long long)absent) - 1;
                    absent &= absent - 1ull;
                    float4* z = reinterpret_cast<float4*>(dst + (u0 + u) * kChunk);
                    const float4 zero = make_float4(0.f, 0.f, 0.f, 0.f);
                    z[0] = zero;
                    z[1] = zero;
                    z[2] = zero;
                    z[3] = zero;
                }
                uint64_t m = pm;
                while (m) {
                    const int u = __ffsll((long long)m) - 1;
                    const int rl = __ffsll((long long)~(m >> u)) - 1;
                    const int x = x0 + u;
                    const bool lw = (x >> 6) == w0;
                    const int64_t r = (int64_t)(lw ? oa : ob) + __popcll((lw ? ua : ub) & ((1ull << (x & 63)) - 1ull));
                    const unsigned bytes = (unsigned)(rl * kChunk * sizeof(float));
                    bar_add_tx(bar, bytes);
                    copy_g2s(dst + (u0 + u) * kChunk, ipool + it.ibase + r * kChunk, bytes, bar);
                    m &= ~(((1ull << rl) - 1ull) << u);
                }
            }
        }
        bar_arrive(bar);
    }
    // output slots of the tile cells of a sparse next layout
    if (!it.dense_out && sw < nj * kT) {
        const int j = sw / kT, rr = sw - j * kT;
        const int s = kNB * k + j;
        if (s >= kFirst) {
            const int zo = out_of(s);
            int* orow = &S.orank[slot][j][rr * kT];
            uint64_t uw = 0ull;
            uint32_t ow = 0u;
            if (rr < it.er) {
                const int64_t row = (int64_t)rowpart(P.ar, it.tr0 + rr, ny) + rowpart(a2, zo, ny);
                const int64_t wi = (int64_t)it.b * G.RW + row * G.W + (it.tx0 >> 6);
                uw = P.out.ubits[wi];
                ow = P.out.woff[wi];
            }
#pragma unroll
            for (int i = 0; i < kT; i++) {
                const int bit = (it.tx0 + i) & 63;  // the 16 cells share one bitmap word
                const bool has = i < it.ex && ((uw >> bit) & 1ull);
                orow[i] = has ? (int)(ow + __popcll(uw & ((1ull << bit) - 1ull))) : -1;
            }
        }
    }
}

template <bool kLim, bool kA0X, int kCodec>
__global__ void __launch_bounds__(kNT, 1) k_gt3(Gt3Args P)
{
    extern __shared__ __align__(16) unsigned char smraw[];
    Gt3Smem& S = *reinterpret_cast<Gt3Smem*>(smraw);
    const GridGeom& G = P.G;
    if (aborted(G.abort)) return;
    const int tid = threadIdx.x;
    const int lane = tid & 31;
    const bool stager = tid >= kNY;   // warps 12-15: stage the next batch during sweep 1
    const int sl = tid - kNY;         // staging lane 0..127
    const int ar = P.ar, a2 = P.ax[2];
    const int n2 = G.n[a2];
    const int nsteps = n2 + kFirst;       // planes streamed per item (3 before, 2 after)
    const int nbatch = (nsteps + kNB - 1) / kNB;
    const int64_t nwork = 4 * P.item_base[G.nb];
    const int64_t str_r = P.stride[ar], str_2 = P.stride[a2];
    // staged offsets of a position along sweep axis 0 / 1 (in floats)
    constexpr int kS0 = kA0X ? kChunk : kRP;
    constexpr int kS1 = kA0X ? kRP : kChunk;
    // the same for the scale table (one float per staged cell)
    constexpr int kC0 = kA0X ? 1 : kSP;
    constexpr int kC1 = kA0X ? kSP : 1;

    if (tid == 0) {
        // one arrival per staging thread
        bar_init(&S.bar[0], kNS);
        bar_init(&S.bar[1], kNS);
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
        S.abort = 0;
        S.pref = 0;
        S.work = (long long)atomicAdd(&P.ctr->work_next, 1ull);
    }
    unsigned gb = 0;   // batches staged by this CTA before the current item (barrier phases)
    unsigned ni = 0;   // items taken by this CTA (parity selects the run and row tables)
    float msum = 0.0f, mcomp = 0.0f;  // Kahan-compensated FP32 mass of this thread

    for (;; ni++) {
        __syncthreads();
        const int64_t w = S.work;
        if (w >= nwork || S.abort) break;
        const bool pref = S.pref != 0;
        const int ti = (int)(ni & 1u);
        const Item it = decode_item(P, w);
        const int64_t okeep = (int64_t)P.out.base[it.b];
        using T = typename Codec<kCodec>::T;
        T* opool = static_cast<T*>(P.out.pool);
        if (!pref) item_tables(P, S, it, ti, tid);
        if (tid < 3 * kChunk) {
            // sweep constants of the item's 16 velocity cells (v = vx + 4 vy, vz = q)
            const int j = tid >> 4, l = tid & 15;
            const int d = P.ax[j];
            const int bc = d == 0 ? it.b % G.nbx : (d == 1 ? (it.b / G.nbx) % G.nby : it.b / (G.nbx * G.nby));
            const int wi = d == 0 ? (l & 3) : (d == 1 ? (l >> 2) : it.q);
            S.kc[j][l] = P.walk[d * P.nvmax + bc * 4 + wi];
        } else if (tid == 64) {
            S.next = (long long)atomicAdd(&P.ctr->work_next, 1ull);
        }
        __syncthreads();  // per-item tables ready
        if (tid == 0) {
            S.pref = 0;
            S.work = S.next;
        }
        const bool up0 = S.kc[0][0].w != 0.0f, up1 = S.kc[1][0].w != 0.0f;
        auto out_of = [&](int s) { return it.up2 ? s - kFirst : n2 + 4 - s; };

        // ---- sweep-2 state of this thread: two tile cells, one vx row of the chunk ----
        const int zq = tid & 3;             // vy of the thread's vx row
        const int zc = tid >> 2;            // tile cells zc and zc + 128
        const int zcx = zc & 15, zcr = zc >> 4;
        const bool zv0 = zcx < it.ex && zcr < it.er, zv1 = zcx < it.ex && zcr + 8 < it.er;
        const int zoff = (kHalo + zcr) * kRP + (kHalo + zcx) * kChunk + 4 * zq;
        const int64_t zcell = (int64_t)(it.tx0 + zcx) + (int64_t)(it.tr0 + zcr) * str_r;  // at plane 0
        Walk2<kLim> zw[4];
#pragma unroll
        for (int i = 0; i < 4; i++) zw[i].reset();
        WalkConst2 kz;
        {
            const float4 c = S.kc[2][4 * zq];  // the streamed axis is not x: equal over vx
            kz.g = make_float2(c.x, c.x);
            kz.A = make_float2(c.y, c.y);
            kz.B = make_float2(c.z, c.z);
        }

        if (stager && !pref) stage_batch<kCodec, kA0X>(P, S, it, ti, 0, gb, sl);
        int k = 0;
        for (; k < nbatch; k++) {
            const unsigned slot = (gb + k) & 1u;
            const unsigned parity = ((gb + k) >> 1) & 1u;
            if (P.report_late && tid == 0 && !bar_test(&S.bar[slot], parity)) atomicOr(&P.ctr->error, 4);
            if (!bar_wait_bounded(&S.bar[slot], parity)) {
                atomicOr(&P.ctr->error, 4);
                S.abort = 1;
            }
            float* B = S.buf[slot][0];
            const int nj = min(kNB, nsteps - kNB * k);
            // sweep 0 along axis 0 on the halo lines that sweep 1 reads
            if (tid < kNX) {
                const int j = tid / (kLines * 8), rem = tid - j * (kLines * 8);
                const int line = rem >> 3, l0 = 2 * (rem & 7);
                if (j < nj) {
                    const float4 c0 = S.kc[0][l0], c1 = S.kc[0][l0 + 1];
                    const WalkConst2 kx{make_float2(c0.x, c1.x), make_float2(c0.y, c1.y), make_float2(c0.z, c1.z)};
                    float* p = B + j * kPS + (line + (up1 ? 0 : 1)) * kS1 + l0;
                    // 16-bit storage: chunk scales of the line's cells
                    const float* ps = scales_of(S) + (slot * kNB + j) * kE * kSP + (line + (up1 ? 0 : 1)) * kC1;
                    // the two staged values of position m: FP32, or two 16-bit codes in the
                    // upper half of the cell's slot
                    // packed codes of the line (sweep 0 along x), see stage_batch
                    const uint32_t* pc = reinterpret_cast<const uint32_t*>(
                                             B + j * kPS + (line + (up1 ? 0 : 1)) * kRP + (up0 ? kCodesHi : 0)) +
                                         (l0 >> 1);
                    auto in = [&](int m) -> float2 {
                        if constexpr (kCodec == 0) {
                            return lds2(p + m * kS0);
                        } else {
                            const float sc = ps[m * kC0];
                            const uint32_t w = kA0X ? pc[m * (kChunk / 2)]
                                                    : reinterpret_cast<const uint32_t*>(p - l0 + m * kS0)[8 + (l0 >> 1)];
                            return dec2<kCodec>(w, make_float2(sc, sc));
                        }
                    };
                    Walk2<kLim> wk;
                    wk.reset();
                    if (up0) {
#pragma unroll
                        for (int m = 0; m < kLines; m++) {
                            const float2 r = wk.push(in(m), kx);
                            if (m >= 5) sts2(p + (m - 2) * kS0, r);
                        }
                    } else {
#pragma unroll
                        for (int m = 0; m < kLines; m++) {
                            const float2 r = wk.push(in(kLines - m), kx);
                            if (m >= 5) sts2(p + (kLines + 2 - m) * kS0, r);
                        }
                    }
                }
            }
            __syncthreads();  // sweep 0 complete; the buffer of batch k-1 is free
            if (S.abort) break;
            if (stager) {
                if (k + 1 < nbatch) {
                    stage_batch<kCodec, kA0X>(P, S, it, ti, k + 1, gb + k + 1, sl);
                } else {
                    // last batch: stage the first batch of the next item
                    const int64_t wn = S.next;
                    if (wn < nwork) {
                        const Item nx = decode_item(P, wn);
                        item_tables(P, S, nx, ti ^ 1, tid);
                        asm volatile("bar.sync 1, %0;\n" ::"n"(kNS) : "memory");
                        stage_batch<kCodec, kA0X>(P, S, nx, ti ^ 1, 0, gb + nbatch, sl);
                        if (sl == 0) S.pref = 1;
                    }
                }
            } else {
                // sweep 1 along axis 1 on the tile lines
                const int j = tid >> 7, rem = tid & 127;
                const int line = rem >> 3, l0 = 2 * (rem & 7);
                if (j < nj) {
                    const float4 c0 = S.kc[1][l0], c1 = S.kc[1][l0 + 1];
                    const WalkConst2 ky{make_float2(c0.x, c1.x), make_float2(c0.y, c1.y), make_float2(c0.z, c1.z)};
                    float* p = B + j * kPS + (kHalo + line) * kS0 + l0;
                    Walk2<kLim> wk;
                    wk.reset();
                    if (up1) {
#pragma unroll
                        for (int m = 0; m < kLines; m++) {
                            const float2 r = wk.push(lds2(p + m * kS1), ky);
                            if (m >= 5) sts2(p + (m - 2) * kS1, r);
                        }
                    } else {
#pragma unroll
                        for (int m = 0; m < kLines; m++) {
                            const float2 r = wk.push(lds2(p + (kLines - m) * kS1), ky);
                            if (m >= 5) sts2(p + (kLines + 2 - m) * kS1, r);
                        }
                    }
                }
            }
            // the in-place writes of this batch precede the bulk copies that refill the
            // buffer two batches on
            fence_async_smem();
            // sweep 1 complete.  The sweep-1 warps do not wait for the staging warps, whose
            // bulk-copy issue can outlast sweep 1: they arrive on barrier 2 and wait among
            // themselves (barrier 3); the staging warps wait on barrier 2 for them
            if (stager) {
                asm volatile("bar.sync 2, %0;\n" ::"n"(kNC) : "memory");
            } else {
                asm volatile("bar.arrive 2, %0;\n" ::"n"(kNC) : "memory");
                asm volatile("bar.sync 3, %0;\n" ::"n"(kNY) : "memory");
            }
            // sweep 2: push the batch's planes through the streamed windows and emit
            auto zplane = [&](int j) {
                const int s = kNB * k + j;
                const float* src = B + j * kPS + zoff;
                const float4 y0 = *reinterpret_cast<const float4*>(src);
                const float4 y1 = *reinterpret_cast<const float4*>(src + 8 * kRP);
                const float2 r00 = zw[0].push(make_float2(y0.x, y0.y), kz);
                const float2 r01 = zw[1].push(make_float2(y0.z, y0.w), kz);
                const float2 r10 = zw[2].push(make_float2(y1.x, y1.y), kz);
                const float2 r11 = zw[3].push(make_float2(y1.z, y1.w), kz);
                if (s < kFirst) return;
                const int zo = out_of(s);
                int64_t rk0, rk1;
                if (it.dense_out) {
                    const int64_t c = zcell + (int64_t)zo * str_2;
                    rk0 = zv0 ? c : -1;
                    rk1 = zv1 ? c + 8 * str_r : -1;
                } else {
                    const int* orow = &S.orank[slot][j][0];
                    rk0 = zv0 ? orow[zc] : -1;
                    rk1 = zv1 ? orow[zc + 128] : -1;
                }
                float psum = 0.0f;
                bool keep0 = false, keep1 = false;
                // 16-bit storage: the scale of each of the two cells' chunk, from the largest
                // magnitude over the four threads (vx rows) of the cell
                ChunkScale cs0{1.0f, 1.0f}, cs1{1.0f, 1.0f};
                if constexpr (kCodec != 0) {
                    cs0 = chunk_scale(group_max<4>(
                        fmaxf(fmaxf(fabsf(r00.x), fabsf(r00.y)), fmaxf(fabsf(r01.x), fabsf(r01.y)))));
                    cs1 = chunk_scale(group_max<4>(
                        fmaxf(fmaxf(fabsf(r10.x), fabsf(r10.y)), fmaxf(fabsf(r11.x), fabsf(r11.y)))));
                }
                // store one vx row (4 values) of a cell; v0, v1 become the values the state
                // now holds (16-bit storage: the codes decoded)
                auto store = [&](int64_t rk, float2& v0, float2& v1, const ChunkScale& cs) {
                    T* dst = opool + it.obase + rk * kChunk + 4 * zq;
                    if constexpr (kCodec == 0) {
                        *reinterpret_cast<float4*>(dst) = make_float4(v0.x, v0.y, v1.x, v1.y);
                    } else {
                        const float2 inv = make_float2(cs.inv, cs.inv), sc = make_float2(cs.s, cs.s);
                        const uint32_t w0 = enc2<kCodec>(v0, inv), w1 = enc2<kCodec>(v1, inv);
                        *reinterpret_cast<uint2*>(dst) = make_uint2(w0, w1);
                        if (zq == 0) P.out.scale[it.obase / kChunk + rk] = cs.s;
                        v0 = dec2<kCodec>(w0, sc);
                        v1 = dec2<kCodec>(w1, sc);
                    }
                };
                if (rk0 >= 0) {
                    float2 v0 = r00, v1 = r01;
                    store(rk0, v0, v1, cs0);
                    psum += (v0.x + v0.y) + (v1.x + v1.y);
                    keep0 = fmaxf(fmaxf(v0.x, v0.y), fmaxf(v1.x, v1.y)) >= P.thr;
                }
                if (rk1 >= 0) {
                    float2 v0 = r10, v1 = r11;
                    store(rk1, v0, v1, cs1);
                    psum += (v0.x + v0.y) + (v1.x + v1.y);
                    keep1 = fmaxf(fmaxf(v0.x, v0.y), fmaxf(v1.x, v1.y)) >= P.thr;
                }
                // per-chunk keep flags: the four threads of a cell vote
                const unsigned b0 = __ballot_sync(0xffffffffu, keep0);
                const unsigned b1 = __ballot_sync(0xffffffffu, keep1);
                if (zq == 0) {
                    if ((b0 >> (lane & ~3)) & 0xfu) P.keepq[(okeep + rk0) * 4 + it.q] = 1;
                    if ((b1 >> (lane & ~3)) & 0xfu) P.keepq[(okeep + rk1) * 4 + it.q] = 1;
                }
                const float y = psum - mcomp;
                const float t = msum + y;
                mcomp = (t - msum) - y;
                msum = t;
            };
            if (nj == kNB) {
#pragma unroll
                for (int j = 0; j < kNB; j++) zplane(j);
            } else {
                for (int j = 0; j < nj; j++) zplane(j);
            }
        }
        if (S.abort) {
            // leave no bulk copy in flight: the batch whose wait ran out is the only one
            // staged and not yet complete
            if (tid == 0 && k < nbatch) bar_wait_bounded(&S.bar[(gb + k) & 1u], ((gb + k) >> 1) & 1u);
            break;
        }
        gb += (unsigned)nbatch;
    }
    double m = (double)msum;
    for (int o = 16; o > 0; o >>= 1) m += __shfl_xor_sync(0xffffffffu, m, o);
    if (lane == 0 && m != 0.0) atomicAdd(&P.ctr->mass, m);
    __syncthreads();
    if (P.cta_done && tid == 0) P.cta_done[blockIdx.x] = now_ns();
}

template <bool kLim, bool kA0X, int kCodec>
vl_status launch_gt3(Grid* g, const Gt3Args& P)
{
    auto kern = k_gt3<kLim, kA0X, kCodec>;
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_bytes<kCodec>());
    int nsm = 0;
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, g->dev.device);
    Gt3Args Q = P;
    if (nsm > kMaxCtas) Q.cta_done = nullptr;
    g->cta_count = Q.cta_done ? nsm : 0;
    g->cta_groups = 1;
    kern<<<nsm, kNT, smem_bytes<kCodec>(), g->stream>>>(Q);
    note_launch();
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(g, e, "plane-batched fused sweep launch");
    return VL_OK;
}

inline int nblocks_of(int64_t n, int t) { return (int)((n + t - 1) / t); }

}  // namespace

bool gt3_applies(const Grid* g, const StepArgs& a)
{
    if (a.ghost != 3) return false;
    if (a.order[2] == 0) return false;  // streamed axis must not be x
    // every velocity block moves one way along each axis
    for (int d = 0; d < 3; d++)
        for (int bi = 0; bi < g->vmesh.nv[d] / 4; bi++) {
            const double lo = g->vmesh.vmin[d] + (4 * bi + 0.5) * g->vmesh.dv[d];
            const double hi = g->vmesh.vmin[d] + (4 * bi + 3.5) * g->vmesh.dv[d];
            if ((lo * a.c_scale[d] >= 0.0) != (hi * a.c_scale[d] >= 0.0)) return false;
        }
    return true;
}

int64_t gt3_tiles(const Grid* g, const StepArgs& a)
{
    const int ar = a.order[0] == 0 ? a.order[1] : a.order[0];
    return (int64_t)((g->geom.n[0] + kT - 1) / kT) * ((g->geom.n[ar] + kT - 1) / kT);
}

vl_status run_gt3(Grid* g, const StepArgs& a)
{
    const GridGeom& G = g->geom;
    Layout& A = g->lay[g->cur];
    Layout& B = g->lay[1 - g->cur];
    const int ar = a.order[0] == 0 ? a.order[1] : a.order[0];
    const int ntile0 = (G.n[0] + kT - 1) / kT;
    const int ntile1 = (G.n[ar] + kT - 1) / kT;
    const int64_t ntiles = (int64_t)ntile0 * ntile1;
    if (ntiles > 0xffffffffLL) return fail(g, VL_EINVAL, "fused form: too many tiles");
    const int64_t need = ntiles * G.nb;
    vl_status wst = fused_worklist_alloc(g, a);
    if (wst != VL_OK) return wst;
    if (need > g->ntiles_alloc) return fail(g, VL_EINVAL, "fused form: work list too small");
    TileArgs T;
    T.G = G;
    T.ubits = B.ubits;
    T.ax[0] = 0;
    T.ax[1] = ar;
    T.ax[2] = a.order[2];
    T.ntile0 = ntile0;
    T.ntile1 = ntile1;
    T.ty = kT;
    launch_tile_list(g, T, need, ntiles);

    Gt3Args P;
    P.G = G;
    P.in = A.view();
    P.out = B.view();
    for (int j = 0; j < 3; j++) P.ax[j] = a.order[j];
    P.ar = ar;
    P.stride[0] = 1;
    P.stride[1] = G.n[0];
    P.stride[2] = (int64_t)G.n[0] * G.n[1];
    P.walk = a.walk;
    P.nvmax = a.nvmax;
    P.thr = (float)g->threshold;
    P.ntile0 = ntile0;
    P.items = g->items;
    P.item_base = g->item_base;
    P.keepq = B.keepq;
    P.ctr = a.ctr;
    P.report_late = fault_requested("timeout") ? 1 : 0;
    P.cta_done = a.stamp_ctas ? g->cta_done : nullptr;
    record_sweep_event(a.ev0, g->stream, a.ev_node);
    const bool a0x = a.order[0] == 0;
    vl_status st = VL_OK;
    with_codec(g->codec, [&](auto c) {
        constexpr int kc = decltype(c)::value;
        if (a0x) st = a.limiter ? launch_gt3<true, true, kc>(g, P) : launch_gt3<false, true, kc>(g, P);
        else st = a.limiter ? launch_gt3<true, false, kc>(g, P) : launch_gt3<false, false, kc>(g, P);
    });
    record_sweep_event(a.ev1, g->stream, a.ev_node);
    (void)nblocks_of;
    return st;
}

}  // namespace vlgt
