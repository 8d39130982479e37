// sweep3.cu -- the classical ("3-pass") translation of libvlgt: one kernel launch per
// Cartesian direction, each reading and writing the whole phase space once (the
// single-GPU analogue of the paper's per-direction ghost update, advection and remote
// contribution, Section 2.1 / Fig. 1).
//
// Pass 1 reads the current layout (present blocks only) and writes every slot of the
// next layout (the 27-cell union); passes 2 and 3 update the next layout in place.  A
// walk runs along one periodic pencil from its upwind end with the sliding-window PPM
// remap.  The vector kernel (k_pass4) gives a thread one vx row of a velocity chunk
// (four walks as two packed pairs, 16-byte accesses) and a CTA item 16 pencils of one
// block id: one CTA per (block id, pencil group) on a dense state, a persistent grid over
// a device-built list of the non-empty pairs on a sparse one.  The scalar kernel (k_pass)
// gives a thread one velocity cell, for blocks whose cells walk in both directions.  The
// last pass also raises the per-chunk keep flags of the sparsity rule (set-only: the
// flags are cleared before the step) and sums the mass.
#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>

#include "grid.h"

namespace vlgt {

namespace {

constexpr int kPencils = 4;                 // pencils per CTA
constexpr int kThreads3 = kPencils * 64;    // one thread per (pencil, velocity cell)
constexpr int kMaxLine = 1024;              // longest pencil held in shared memory

struct PassArgs {
    GridGeom G;
    LayoutView in, out;
    int dim;            // physical axis of this pass
    int check_keep_in;  // 1: read only present blocks of `in`
    int in_is_out;      // 1: `in` and `out` are the same layout (passes 2 and 3, in place)
    double cs;          // dt / dx_dim
    double vmin, dv;    // velocity mesh along dim
    int last;           // last pass: keep flags and mass
    float thr;
    uint8_t* keepq;
    StepCounters* ctr;
    int64_t groups;     // pencil groups per block id
    // vector kernel, list mode: work list of the (block id, pencil group) pairs that hold
    // any slot of the next layout (items[0 .. item_base[nb]) = b * groups + group), taken
    // by a persistent grid through the counter `next`
    const uint32_t* items;
    const int64_t* item_base;
    unsigned long long* next;
    uint64_t* cta_done;  // optional, list mode [gridDim.x]: %globaltimer when the CTA ran out of work
};

// physical coordinates of pencil p, position i along dim
__device__ __forceinline__ void pencil_cell(const GridGeom& G, int dim, int64_t p, int i, int& x,
                                            int64_t& row)
{
    if (dim == 0) {
        x = i;
        row = p;  // row = y + ny*z
    } else if (dim == 1) {
        x = (int)(p % G.n[0]);
        int64_t z = p / G.n[0];
        row = i + (int64_t)G.n[1] * z;
    } else {
        x = (int)(p % G.n[0]);
        int64_t y = p / G.n[0];
        row = y + (int64_t)G.n[1] * i;
    }
}

template <bool kLim, int kCodec>
__global__ void __launch_bounds__(kThreads3) k_pass(PassArgs P)
{
    using C = Codec<kCodec>;
    using T = typename C::T;
    __shared__ int s_rin[kPencils][kMaxLine];
    __shared__ int s_rout[kPencils][kMaxLine];
    __shared__ int s_any[kPencils];
    // 16-bit storage: largest |new value| per (pencil, chunk, cell) as float bits,
    // [kPencils][4][nd].  The velocity cells of a chunk may walk in opposite directions
    // here (a block straddling v = 0), so a chunk's 16 new values appear at different
    // times: a first walk finds their maximum, a second one encodes and stores.
    extern __shared__ unsigned s_cmax[];
    const GridGeom& G = P.G;
    if (aborted(G.abort)) return;
    const int b = (int)(blockIdx.x / P.groups);
    const int64_t grp = blockIdx.x % P.groups;
    const int nd = G.n[P.dim];
    const int64_t npen = G.N / nd;
    if (P.out.cnt[b] == 0) return;

    // ranks of every cell of the CTA's pencils in both layouts
    if (threadIdx.x < kPencils) s_any[threadIdx.x] = 0;
    if constexpr (kCodec != 0)
        for (int t = threadIdx.x; t < kPencils * 4 * nd; t += blockDim.x) s_cmax[t] = 0u;
    __syncthreads();
    for (int t = threadIdx.x; t < kPencils * nd; t += blockDim.x) {
        int k = t / nd, i = t - k * nd;
        int64_t p = grp * kPencils + k;
        int ri = -1, ro = -1;
        if (p < npen) {
            int x;
            int64_t row;
            pencil_cell(G, P.dim, p, i, x, row);
            ri = (int)cell_rank(P.in, G, b, x, row, P.check_keep_in != 0);
            ro = (int)cell_rank(P.out, G, b, x, row, false);
        }
        s_rin[k][i] = ri;
        s_rout[k][i] = ro;
        if (ro >= 0) s_any[k] = 1;
    }
    __syncthreads();
    const int k = threadIdx.x >> 6;
    const int v = threadIdx.x & 63;
    // nothing of this pencil is in the next layout (warp-uniform); with 16-bit storage
    // the pencil's threads stay for the CTA's barriers and skip the walks
    const bool active = s_any[k] != 0;
    if (kCodec == 0 && !active) return;

    const int q = v >> 4, l = v & 15;
    int bc[3] = {b % G.nbx, (b / G.nbx) % G.nby, b / (G.nbx * G.nby)};
    int within[3] = {v & 3, (v >> 2) & 3, v >> 4};
    int iv = bc[P.dim] * 4 + within[P.dim];
    const WalkConst kc = walk_const((P.vmin + (iv + 0.5) * P.dv) * P.cs);
    const bool up = kc.up != 0;
    // the warp's velocity cells move the same way unless the block straddles v_d = 0
    const bool uni = __all_sync(0xffffffffu, up) || __all_sync(0xffffffffu, !up);

    // chunk indices of cell rank 0 of this chunk row in both layouts (16-bit storage
    // keeps one scale per chunk, indexed like the chunks)
    const int64_t cin = (int64_t)P.in.base[b] * 4 + (int64_t)q * P.in.cnt[b];
    const int64_t cout = (int64_t)P.out.base[b] * 4 + (int64_t)q * P.out.cnt[b];
    const T* src = static_cast<const T*>(P.in.pool) + cin * kChunk + l;
    T* dst = static_cast<T*>(P.out.pool) + cout * kChunk + l;
    const int* rin = s_rin[k];
    const int* rout = s_rout[k];
    unsigned* cmax = s_cmax + (k * 4 + q) * nd;
    // the walk runs from the upwind end: walking position m is cell m (c >= 0) or
    // cell nd-1-m (c < 0)
    auto cell_at = [&](int m) { return up ? m : nd - 1 - m; };
    auto load = [&](int m) -> float {
        int r = rin[cell_at(m)];
        return r >= 0 ? C::dec(src[(int64_t)r * kChunk], kCodec ? P.in.scale[cin + r] : 1.0f) : 0.0f;
    };
    float msum = 0.0f;
    double mass = 0.0;
    // one walk over the pencil calling emit(mm, res) with the new average of every
    // walking position mm
    auto walk = [&](auto emit) {
        // originals of walking positions 0 and 1, read again by the wrapped tail after
        // they were updated in place
        const float t0 = load(0), t1 = load(1 % nd);
        Walk<kLim> s;
        s.reset();
        int m = -3;
        for (; m < 0; m++) s.push(load(wrapi(m, nd)), kc);
        // main walk, loads batched ahead of the dependent arithmetic
        for (; m + 8 <= nd; m += 8) {
            float a[8];
#pragma unroll
            for (int u = 0; u < 8; u++) a[u] = load(m + u);
#pragma unroll
            for (int u = 0; u < 8; u++) {
                float res = s.push(a[u], kc);
                if (m + u >= 2) emit(m + u - 2, res);
            }
            mass += (double)msum;
            msum = 0.0f;
        }
        for (; m < nd; m++) {
            float res = s.push(load(m), kc);
            if (m >= 2) emit(m - 2, res);
        }
        const float tail[2] = {t0, t1};
#pragma unroll
        for (int u = 0; u < 2; u++, m++) {
            float res = s.push(tail[u], kc);
            if (m >= 2) emit(m - 2, res);
        }
    };
    const float thr = P.thr;
    auto emit = [&](int mm, float res) {  // new average of walking position mm
        int c = cell_at(mm);
        int r = rout[c];
        T code;
        if constexpr (kCodec != 0) {
            const ChunkScale cs = chunk_scale(__uint_as_float(cmax[c]));
            code = C::enc(res, cs.inv);
            res = C::dec(code, cs.s);  // the value the state now holds
        } else {
            code = res;
        }
        if (r >= 0) dst[(int64_t)r * kChunk] = code;
        if (P.last) {
            bool keep = r >= 0 && res >= thr;
            uint8_t* kq = P.keepq + ((int64_t)P.out.base[b] + r) * 4 + q;
            if (uni) {
                unsigned m = __ballot_sync(0xffffffffu, keep);
                unsigned half = (threadIdx.x & 16) ? (m >> 16) : (m & 0xffffu);
                if (half && (threadIdx.x & 15) == 0) *kq = 1;
            } else if (keep) {
                *kq = 1;
            }
            if (r >= 0) msum += res;
        }
    };
    if constexpr (kCodec != 0) {
        if (active)
            walk([&](int mm, float res) {
                const int c = cell_at(mm);
                if (rout[c] >= 0) atomicMax(&cmax[c], __float_as_uint(fabsf(res)));
            });
        __syncthreads();  // every chunk's maximum is complete
        // the second walk reads the codes with the scales they were written with (in
        // place: the new scales replace them only after it)
        if (active) walk(emit);
        __syncthreads();
        for (int t = threadIdx.x; t < kPencils * 4 * nd; t += blockDim.x) {
            const int kk = t / (4 * nd), rem = t - kk * 4 * nd;
            const int qq = rem / nd, c = rem - qq * nd;
            const int r = s_rout[kk][c];
            if (r >= 0)
                P.out.scale[(int64_t)P.out.base[b] * 4 + (int64_t)qq * P.out.cnt[b] + r] =
                    chunk_scale(__uint_as_float(s_cmax[t])).s;
        }
        if (!active) return;
    } else {
        walk(emit);
    }
    if (P.last) {
        mass += (double)msum;
        for (int o = 16; o > 0; o >>= 1) mass += __shfl_xor_sync(0xffffffffu, mass, o);
        if ((threadIdx.x & 31) == 0 && mass != 0.0) atomicAdd(&P.ctr->mass, mass);
    }
}


// ---- vector form: four velocity cells per thread ------------------------------------
// Same walk as k_pass, but a thread owns one vx row (4 cells) of a velocity chunk and
// moves it with 16-byte loads and stores (8-byte in 16-bit storage): four independent
// walks per thread, a quarter of the memory instructions.  A CTA holds 16 pencils, which
// are neighbours along x for the y and z passes, so a warp touches 128 contiguous bytes
// per chunk.  The four cells of a thread share the walking direction: always for the y
// and z passes (they differ only in vx), and for the x pass when no block straddles
// v_x = 0 (the host checks; otherwise it launches k_pass).
constexpr int kPen4 = 16;
constexpr int kThreads4 = kPen4 * 16;
constexpr int kBatch4 = 8;

template <int kCodec>
__device__ __forceinline__ void load4(const typename Codec<kCodec>::T* p, float sc, float (&o)[4])
{
    if constexpr (kCodec == 0) {
        const float4 v = *reinterpret_cast<const float4*>(p);
        o[0] = v.x;
        o[1] = v.y;
        o[2] = v.z;
        o[3] = v.w;
    } else {
        const uint2 raw = *reinterpret_cast<const uint2*>(p);
        const typename Codec<kCodec>::T* h = reinterpret_cast<const typename Codec<kCodec>::T*>(&raw);
#pragma unroll
        for (int i = 0; i < 4; i++) o[i] = Codec<kCodec>::dec(h[i], sc);
    }
}

template <int kCodec>
__device__ __forceinline__ void store4(typename Codec<kCodec>::T* p, const typename Codec<kCodec>::T (&c)[4])
{
    if constexpr (kCodec == 0) {
        *reinterpret_cast<float4*>(p) = make_float4(c[0], c[1], c[2], c[3]);
    } else {
        uint2 raw;
        typename Codec<kCodec>::T* h = reinterpret_cast<typename Codec<kCodec>::T*>(&raw);
#pragma unroll
        for (int i = 0; i < 4; i++) h[i] = c[i];
        *reinterpret_cast<uint2*>(p) = raw;
    }
}

// Any of the bits xlo .. xhi-1 (0 <= xlo < xhi <= nx) set in a bitmap row.
__device__ bool row_has(const uint64_t* rowp, int xlo, int xhi)
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

// flags[b][grp] = 1 when a pencil of group grp (pencils kPen4 grp .. kPen4 grp + kPen4 - 1
// along dim, in pencil_cell's numbering) holds a slot of block id b in the layout
__global__ void k_pass_groups(GridGeom G, const uint64_t* __restrict__ ubits, int dim, int64_t ngroups,
                              uint32_t* __restrict__ flags)
{
    if (aborted(G.abort)) return;
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (int64_t)G.nb * ngroups) return;
    const int b = (int)(i / ngroups);
    const int64_t grp = i - (int64_t)b * ngroups;
    const uint64_t* seg = ubits + (int64_t)b * G.RW;
    const int nd = G.n[dim];
    const int64_t npen = G.N / nd;
    const int64_t p0 = grp * kPen4, p1 = min(p0 + kPen4, npen);
    bool any = false;
    if (dim == 0) {
        // pencils are rows
        for (int64_t row = p0; row < p1 && !any; row++)
            for (int w = 0; w < G.W && !any; w++) any = seg[row * G.W + w] != 0;
    } else {
        // pencil p = x + nx o (o = z along y, y along z): the group is at most two runs of x
        const int nx = G.n[0];
        for (int64_t p = p0; p < p1 && !any;) {
            const int64_t o = p / nx;
            const int xa = (int)(p - o * nx);
            const int xb = (int)min((int64_t)nx, xa + (p1 - p));
            for (int c = 0; c < nd && !any; c++) {
                const int64_t row = dim == 1 ? c + (int64_t)G.n[1] * o : o + (int64_t)G.n[1] * c;
                any = row_has(seg + row * G.W, xa, xb);
            }
            p += xb - xa;
        }
    }
    flags[i] = any ? 1u : 0u;
}

// kLast: the last pass (keep flags and mass, which need the values the state now holds).
// An item is one (block id, group of kPen4 pencils) pair.  kList: a persistent grid takes
// the pairs of the work list and skips batches of positions with no slot; otherwise one
// CTA per pair (a fully dense layout, where every pair is an item).
template <bool kLim, int kCodec, bool kLast, bool kList>
__global__ void __launch_bounds__(kThreads4, 2) k_pass4(PassArgs P)
{
    using C = Codec<kCodec>;
    using T = typename C::T;
    // [kPen4][nd] input ranks and output ranks (passes 2 and 3 work in place and share
    // one table), then (list mode) [kPen4][nw] bitmaps of the cells with an output slot
    extern __shared__ int s_rank4[];
    __shared__ int s_any[kPen4];
    __shared__ long long s_w;
    const GridGeom& G = P.G;
    if (aborted(G.abort)) return;
    // list mode: thread 0 takes the next item's index one item ahead, so that the
    // atomic's latency passes during the current item
    unsigned long long nx = 0;
    if (kList && threadIdx.x == 0) nx = atomicAdd(P.next, 1ull);
    const int nd = G.n[P.dim];
    const int nw = (nd + 31) >> 5;
    const int64_t npen = G.N / nd;
    int* s_rin = s_rank4;
    int* s_rout = P.in_is_out ? s_rank4 : s_rank4 + kPen4 * nd;
    uint32_t* s_slot = reinterpret_cast<uint32_t*>(s_rank4 + (P.in_is_out ? 1 : 2) * kPen4 * nd);
    const int k = threadIdx.x >> 4;        // pencil; a warp holds pencils k and k^1
    const int q = (threadIdx.x >> 2) & 3;  // velocity chunk (vz within the block)
    const int vy = threadIdx.x & 3;        // vx row of the chunk
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    double mass = 0.0;  // last pass: this thread's stored values over all its items
    for (bool first = true;; first = false) {
        int64_t pair = blockIdx.x;
        if constexpr (kList) {
            __syncthreads();  // the previous item's tables are no longer read
            if (threadIdx.x == 0) {
                s_w = (long long)nx;
                nx = atomicAdd(P.next, 1ull);
            }
            if (threadIdx.x < kPen4) s_any[threadIdx.x] = 0;
            __syncthreads();
            const int64_t w = s_w;
            if (w >= P.item_base[G.nb]) break;
            pair = P.items[w];
        } else {
            if (!first) break;
            if (threadIdx.x < kPen4) s_any[threadIdx.x] = 0;
            __syncthreads();
        }
        const int b = (int)(pair / P.groups);
        const int64_t grp = pair - (int64_t)b * P.groups;
        if (P.out.cnt[b] == 0) continue;  // CTA-uniform
        for (int t = threadIdx.x; t < kPen4 * nd; t += blockDim.x) {
            int kk = t / nd, i = t - kk * nd;
            int64_t p = grp * kPen4 + kk;
            int ri = -1, ro = -1;
            if (p < npen) {
                int x;
                int64_t row;
                pencil_cell(G, P.dim, p, i, x, row);
                ro = (int)cell_rank(P.out, G, b, x, row, false);
                ri = P.in_is_out ? ro : (int)cell_rank(P.in, G, b, x, row, P.check_keep_in != 0);
            }
            s_rin[kk * nd + i] = ri;
            if (!P.in_is_out) s_rout[kk * nd + i] = ro;
            if (ro >= 0) s_any[kk] = 1;
        }
        __syncthreads();
        if constexpr (kList) {
            // which cells have an output slot, 32 per ballot
            for (int j = warp; j < kPen4 * nw; j += kThreads4 / 32) {
                const int kk = j / nw, c = ((j - kk * nw) << 5) + lane;
                const unsigned bits = __ballot_sync(0xffffffffu, c < nd && s_rout[kk * nd + c] >= 0);
                if (lane == 0) s_slot[j] = bits;
            }
            __syncthreads();
        }
        if (!s_any[k] && !s_any[k ^ 1]) continue;  // warp-uniform

        const int bc[3] = {b % G.nbx, (b / G.nbx) % G.nby, b / (G.nbx * G.nby)};
        WalkConst kc[4];
    #pragma unroll
        for (int i = 0; i < 4; i++) {
            const int within = P.dim == 0 ? i : (P.dim == 1 ? vy : q);
            const int iv = bc[P.dim] * 4 + within;
            kc[i] = walk_const((P.vmin + (iv + 0.5) * P.dv) * P.cs);
        }
        const bool up = kc[0].up != 0;
        const WalkConst2 kp[2] = {pack_const(kc[0], kc[1]), pack_const(kc[2], kc[3])};
        const bool uni = __all_sync(0xffffffffu, up) || __all_sync(0xffffffffu, !up);

        const int64_t cin = (int64_t)P.in.base[b] * 4 + (int64_t)q * P.in.cnt[b];    // chunk of rank 0
        const int64_t cout = (int64_t)P.out.base[b] * 4 + (int64_t)q * P.out.cnt[b];
        const T* src = static_cast<const T*>(P.in.pool) + cin * kChunk + 4 * vy;
        T* dst = static_cast<T*>(P.out.pool) + cout * kChunk + 4 * vy;
        const int* rin = s_rin + k * nd;
        const int* rout = s_rout + k * nd;
        auto cell_at = [&](int m) { return up ? m : nd - 1 - m; };
        auto load = [&](int m, float (&o)[4]) {
            const int r = rin[cell_at(m)];
            if (r >= 0) {
                load4<kCodec>(src + (int64_t)r * kChunk, kCodec ? P.in.scale[cin + r] : 1.0f, o);
            } else {
                o[0] = o[1] = o[2] = o[3] = 0.0f;
            }
        };
        float t0[4], t1[4];  // originals of walking positions 0 and 1 (the wrapped tail)
        load(0, t0);
        load(1 % nd, t1);

        Walk2<kLim> s[2];  // cells (0, 1) and (2, 3) of the row, packed
        s[0].reset();
        s[1].reset();
        float msum = 0.0f;
        const float thr = P.thr;
        // every lane calls it for the same position; the 4 lanes of a chunk (one vx row each)
        // are consecutive, and in place they have all read the chunk at position m - 2 before
        // the shuffles of that position's call, so its scale may be replaced
        auto push_emit = [&](int m, const float (&a)[4]) {
            float res[4];
            const float2 r01 = s[0].push(make_float2(a[0], a[1]), kp[0]);
            const float2 r23 = s[1].push(make_float2(a[2], a[3]), kp[1]);
            res[0] = r01.x;
            res[1] = r01.y;
            res[2] = r23.x;
            res[3] = r23.y;
            if (m < 2) return;
            const int c = cell_at(m - 2);
            const int r = rout[c];
            T code[4];
            if constexpr (kCodec != 0) {
                const float mx = fmaxf(fmaxf(fabsf(res[0]), fabsf(res[1])), fmaxf(fabsf(res[2]), fabsf(res[3])));
                const ChunkScale cs = chunk_scale(group_max<4>(mx));
    #pragma unroll
                for (int i = 0; i < 4; i++) {
                    code[i] = C::enc(res[i], cs.inv);
                    if constexpr (kLast) res[i] = C::dec(code[i], cs.s);  // the value the state now holds
                }
                if (r >= 0 && vy == 0) P.out.scale[cout + r] = cs.s;
            } else {
    #pragma unroll
                for (int i = 0; i < 4; i++) code[i] = res[i];
            }
            if (r >= 0) store4<kCodec>(dst + (int64_t)r * kChunk, code);
            if constexpr (kLast) {
                const bool keep = r >= 0 && (res[0] >= thr || res[1] >= thr || res[2] >= thr || res[3] >= thr);
                uint8_t* kq = P.keepq + ((int64_t)P.out.base[b] + r) * 4 + q;
                if (uni) {
                    const unsigned bal = __ballot_sync(0xffffffffu, keep);
                    const unsigned nib = (bal >> ((threadIdx.x & 31) & ~3u)) & 0xfu;  // the chunk's 4 rows
                    if (nib && vy == 0) *kq = 1;
                } else if (keep) {
                    *kq = 1;
                }
                if (r >= 0) msum += (res[0] + res[1]) + (res[2] + res[3]);
            }
        };
        // list mode: a batch of positions m .. m+7 is skipped when positions m-10 .. m+7 hold
        // no output slot in any lane's pencil: the walk has then pushed at least 8 zeros, so
        // its state is zero and stays so, and every position the batch would emit has no slot
        auto idle = [&](int m) -> bool {
            bool quiet = false;
            if (m >= 10) {
                const int c0 = up ? m - 10 : nd - m - 8;  // cells c0 .. c0+17
                const uint32_t* mk = s_slot + k * nw;
                const int w0 = c0 >> 5;
                uint64_t v = mk[w0];
                if (w0 + 1 < nw) v |= (uint64_t)mk[w0 + 1] << 32;
                quiet = ((v >> (c0 & 31)) & 0x3ffffull) == 0ull;
            }
            return __all_sync(0xffffffffu, quiet);
        };
        int m = -3;
        for (; m < 0; m++) {
            float a[4];
            load(wrapi(m, nd), a);
            s[0].push(make_float2(a[0], a[1]), kp[0]);
            s[1].push(make_float2(a[2], a[3]), kp[1]);
        }
        if constexpr (kCodec == 0) {
            for (; m + kBatch4 <= nd; m += kBatch4) {
                if (kList && idle(m)) continue;
                float a[kBatch4][4];
    #pragma unroll
                for (int u = 0; u < kBatch4; u++) load(m + u, a[u]);
                // L2 prefetch of the next batch (one lane per chunk row): DRAM keeps working
                // while this batch's arithmetic runs, and the next loads hit L2.  It takes no
                // registers; a distance of one batch measured best (0.88 of the copy
                // bandwidth against 0.76 without, 0.85 at two batches).
                if (vy == 0) {
    #pragma unroll
                    for (int u = 0; u < kBatch4; u++) {
                        const int pm = m + kBatch4 + u;
                        if (pm < nd) {
                            const int r = rin[cell_at(pm)];
                            if (r >= 0) asm volatile("prefetch.global.L2 [%0];" ::"l"(src + (int64_t)r * kChunk));
                        }
                    }
                }
    #pragma unroll
                for (int u = 0; u < kBatch4; u++) push_emit(m + u, a[u]);
                if constexpr (kLast) {
                    mass += (double)msum;
                    msum = 0.0f;
                }
            }
        } else {
            // 16-bit storage: the batch is held as raw codes and scales (3 registers per
            // position instead of 4) and decoded as it is pushed; the next batch's code
            // sectors and scales are prefetched into L2 like the FP32 rows (50.4 against 64.3
            // ms per bfloat16 step without; batches of 12 positions measured 52.6 ms)
            for (; m + kBatch4 <= nd; m += kBatch4) {
                if (kList && idle(m)) continue;
                uint2 raw[kBatch4];
                float sc[kBatch4];
    #pragma unroll
                for (int u = 0; u < kBatch4; u++) {
                    const int r = rin[cell_at(m + u)];
                    raw[u] = r >= 0 ? *reinterpret_cast<const uint2*>(src + (int64_t)r * kChunk) : make_uint2(0u, 0u);
                    sc[u] = r >= 0 ? P.in.scale[cin + r] : 0.0f;
                }
                if (vy == 0) {
    #pragma unroll
                    for (int u = 0; u < kBatch4; u++) {
                        const int pm = m + kBatch4 + u;
                        if (pm < nd) {
                            const int r = rin[cell_at(pm)];
                            if (r >= 0) {
                                asm volatile("prefetch.global.L2 [%0];" ::"l"(src + (int64_t)r * kChunk));
                                asm volatile("prefetch.global.L2 [%0];" ::"l"(P.in.scale + cin + r));
                            }
                        }
                    }
                }
    #pragma unroll
                for (int u = 0; u < kBatch4; u++) {
                    float a[4];
                    const T* h = reinterpret_cast<const T*>(&raw[u]);
    #pragma unroll
                    for (int i = 0; i < 4; i++) a[i] = C::dec(h[i], sc[u]);
                    push_emit(m + u, a);
                }
                if constexpr (kLast) {
                    mass += (double)msum;
                    msum = 0.0f;
                }
            }
        }
        for (; m < nd; m++) {
            float a[4];
            load(m, a);
            push_emit(m, a);
        }
        push_emit(m, t0);
        push_emit(m + 1, t1);
        if constexpr (kLast) mass += (double)msum;
    }
    if constexpr (kLast) {
        for (int o = 16; o > 0; o >>= 1) mass += __shfl_xor_sync(0xffffffffu, mass, o);
        if (lane == 0 && mass != 0.0) atomicAdd(&P.ctr->mass, mass);
    }
    if (kList && P.cta_done && threadIdx.x == 0) {
        uint64_t t;
        asm volatile("mov.u64 %0, %%globaltimer;\n" : "=l"(t));
        P.cta_done[blockIdx.x] = t;
    }
}

}  // namespace

// Work-list buffers for the largest pass: groups of kPen4 pencils x block ids.
vl_status pass_worklist_alloc(Grid* g)
{
    const GridGeom& G = g->geom;
    int64_t need = 0;
    for (int d = 0; d < 3; d++) need = std::max(need, (G.N / G.n[d] + kPen4 - 1) / kPen4 * G.nb);
    return worklist_reserve(g, need);
}

vl_status run_3pass(Grid* g, const StepArgs& a)
{
    const GridGeom& G = g->geom;
    Layout& A = g->lay[g->cur];
    Layout& B = g->lay[1 - g->cur];
    for (int d = 0; d < 3; d++)
        if (G.n[d] > kMaxLine)
            return fail(g, VL_EINVAL, "3-pass form: grid extent above 1024 cells");
    vl_status wst = pass_worklist_alloc(g);
    if (wst != VL_OK) return wst;
    int stamped[3] = {0, 0, 0};  // CTAs of each pass that stamp their finish time
    int nsm = 0;
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, g->dev.device);
    record_sweep_event(a.ev0, g->stream, a.ev_node);
    for (int j = 0; j < 3; j++) {
        int d = a.order[j];
        PassArgs P;
        P.G = G;
        P.in = j == 0 ? A.view() : B.view();
        P.out = B.view();
        P.dim = d;
        P.check_keep_in = j == 0 ? 1 : 0;
        P.in_is_out = j == 0 ? 0 : 1;
        P.cs = a.c_scale[d];
        P.vmin = g->vmesh.vmin[d];
        P.dv = g->vmesh.dv[d];
        P.last = j == 2 ? 1 : 0;
        P.thr = (float)g->threshold;
        P.keepq = B.keepq;
        P.ctr = a.ctr;
        P.items = nullptr;
        P.item_base = nullptr;
        P.next = &a.ctr->pass_next[j];
        P.cta_done = nullptr;
        int64_t npen = G.N / G.n[d];
        // the vector kernel needs one walking direction per vx row: along x, no block
        // may straddle v_x = 0.  With 16-bit storage the four rows of a chunk must also
        // walk together (they share the chunk's scale), which along y needs the same
        bool vec = true;
        if (d == 0 || (d == 1 && g->codec)) {
            const int nbd = d == 0 ? G.nbx : G.nby;
            for (int bi = 0; bi < nbd && vec; bi++) {
                const double lo = P.vmin + (4 * bi + 0.5) * P.dv, hi = P.vmin + (4 * bi + 3.5) * P.dv;
                if ((lo >= 0.0) != (hi >= 0.0)) vec = false;
            }
        }
        const int per_cta = vec ? kPen4 : kPencils;
        P.groups = (npen + per_cta - 1) / per_cta;
        int64_t nblocks = P.groups * G.nb;
        if (nblocks > 0x7fffffffLL) return fail(g, VL_EINVAL, "3-pass form: grid too large");
        // a sparse state (under 3/4 of the (cell, block id) pairs present): a list of the
        // (block id, pencil group) pairs that hold any slot of the next layout, for a
        // persistent grid; a dense one takes every pair, one CTA each
        const bool listed = vec && g->present < G.N * (int64_t)G.nb / 4 * 3;
        // rank tables (one when the pass works in place) and, listed, the slot bitmaps
        const int smem4 =
            ((P.in_is_out ? 1 : 2) * kPen4 * G.n[d] + (listed ? kPen4 * ((G.n[d] + 31) / 32) : 0)) * (int)sizeof(int);
        if (listed) {
            k_pass_groups<<<(unsigned)((nblocks + 255) / 256), 256, 0, g->stream>>>(G, B.ubits, d, P.groups,
                                                                                    g->tile_flags);
            note_launch();
            launch_items_from_flags(g, P.groups, true);
            P.items = g->items;
            P.item_base = g->item_base;
        }
        with_codec(g->codec, [&](auto c) {
            constexpr int kc = decltype(c)::value;
            if (vec) {
                auto pick = [&](auto list_tag) {
                    constexpr bool kL = decltype(list_tag)::value;
                    return a.limiter ? (P.last ? k_pass4<true, kc, true, kL> : k_pass4<true, kc, false, kL>)
                                     : (P.last ? k_pass4<false, kc, true, kL> : k_pass4<false, kc, false, kL>);
                };
                auto kern = listed ? pick(std::true_type{}) : pick(std::false_type{});
                if (smem4 > 48 * 1024) cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem4);
                int per_sm = 0;
                cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kThreads4, smem4);
                const int64_t nct = listed ? std::min<int64_t>(nblocks, (int64_t)nsm * std::max(per_sm, 1)) : nblocks;
                // each pass of a listed step stamps its CTAs into its own third of the
                // array (the idle tail of the persistent grid, reported as tail_ms)
                if (listed && a.stamp_ctas && 3 * nct <= kMaxCtas) {
                    P.cta_done = g->cta_done + j * nct;
                    stamped[j] = (int)nct;
                }
                kern<<<(unsigned)nct, kThreads4, smem4, g->stream>>>(P);
            } else {
                auto kern = a.limiter ? k_pass<true, kc> : k_pass<false, kc>;
                // 16-bit storage: per-chunk maxima of the pencils
                const int smem = kc ? kPencils * 4 * G.n[d] * (int)sizeof(unsigned) : 0;
                if (smem > 0) cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
                kern<<<(unsigned)nblocks, kThreads3, smem, g->stream>>>(P);
            }
        });
        note_launch();
    }
    record_sweep_event(a.ev1, g->stream, a.ev_node);
    // tails are reported when every pass stamped (all three listed, equal grids)
    const bool all = stamped[0] > 0 && stamped[0] == stamped[1] && stamped[1] == stamped[2];
    g->cta_count = all ? stamped[0] : 0;
    g->cta_groups = all ? 3 : 1;
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(g, e, "3-pass sweep launch");
    return VL_OK;
}

}  // namespace vlgt
