// layout.cu -- sparse velocity-space bookkeeping of libvlgt: block-set union (27-cell
// dilation of the presence bitmaps), slot indexing (segmented scans), the sparsity rule
// (keep flags -> presence bitmaps, FP64 dropped mass), conversion from and to per-cell
// block lists, and FP64 velocity moments.
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "grid.h"

namespace vlgt {

namespace {

constexpr int kScanThreads = 1024;

__device__ __forceinline__ uint32_t warp_incl_scan(uint32_t x, int lane)
{
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    return x;
}

__device__ __forceinline__ unsigned long long warp_incl_scan64(unsigned long long x, int lane)
{
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        unsigned long long y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    return x;
}

// Exclusive scan of each segment of seg_len counts; one CTA per segment.
__global__ void k_seg_scan(const uint32_t* __restrict__ in, uint32_t* __restrict__ out,
                           uint32_t* __restrict__ seg_total, int64_t seg_len, const int* abort)
{
    if (aborted(abort)) return;
    __shared__ uint32_t wsum[32];
    const int64_t seg = blockIdx.x;
    const uint32_t* src = in + seg * seg_len;
    uint32_t* dst = out + seg * seg_len;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    uint32_t carry = 0;
    for (int64_t start = 0; start < seg_len; start += blockDim.x) {
        int64_t i = start + threadIdx.x;
        uint32_t v = i < seg_len ? src[i] : 0u;
        uint32_t x = warp_incl_scan(v, lane);
        if (lane == 31) wsum[warp] = x;
        __syncthreads();
        if (warp == 0) {
            uint32_t w = lane < nw ? wsum[lane] : 0u;
            w = warp_incl_scan(w, lane);
            wsum[lane] = w;
        }
        __syncthreads();
        uint32_t pre = carry + (warp > 0 ? wsum[warp - 1] : 0u);
        if (i < seg_len) dst[i] = pre + x - v;
        carry += wsum[nw - 1];
        __syncthreads();
    }
    if (threadIdx.x == 0) seg_total[seg] = carry;
}

// base[s] = sum of seg_total[0..s), base[nseg] = grand total (64-bit); one CTA.
__global__ void k_base_scan(const uint32_t* __restrict__ seg_total, int64_t* __restrict__ base,
                            int64_t nseg, const int* abort)
{
    if (aborted(abort)) return;
    __shared__ unsigned long long wsum[32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    unsigned long long carry = 0;
    for (int64_t start = 0; start < nseg; start += blockDim.x) {
        int64_t i = start + threadIdx.x;
        unsigned long long v = i < nseg ? seg_total[i] : 0ull;
        unsigned long long x = warp_incl_scan64(v, lane);
        if (lane == 31) wsum[warp] = x;
        __syncthreads();
        if (warp == 0) {
            unsigned long long w = lane < nw ? wsum[lane] : 0ull;
            w = warp_incl_scan64(w, lane);
            wsum[lane] = w;
        }
        __syncthreads();
        unsigned long long pre = carry + (warp > 0 ? wsum[warp - 1] : 0ull);
        if (i < nseg) base[i] = (int64_t)(pre + x - v);
        carry += wsum[nw - 1];
        __syncthreads();
    }
    if (threadIdx.x == 0) base[nseg] = (int64_t)carry;
}

__device__ __forceinline__ uint64_t word_mask(int nx, int w)
{
    int last = nx - 1;
    if (w < (last >> 6)) return ~0ull;
    int top = last & 63;
    return top == 63 ? ~0ull : ((1ull << (top + 1)) - 1ull);
}

// One word of a row dilated by one cell along x with periodic wrap.
__device__ __forceinline__ uint64_t xdilate(const uint64_t* row, int W, int nx, int w)
{
    uint64_t cur = row[w];
    uint64_t prev = w > 0 ? row[w - 1] : 0ull;
    uint64_t next = (w + 1 < W) ? row[w + 1] : 0ull;
    uint64_t left = (cur << 1) | (prev >> 63);   // bit x receives bit x-1
    uint64_t right = (cur >> 1) | (next << 63);  // bit x receives bit x+1
    int last = nx - 1;
    if (w == 0) left |= (row[last >> 6] >> (last & 63)) & 1ull;
    if (w == (last >> 6)) right |= (row[0] & 1ull) << (last & 63);
    return cur | left | right;
}

// next.ubits = union of cur.kbits over the 3x3x3 periodic neighbourhood (a block can
// only arrive from a cell at most one step away along each axis, since |c| <= 1 per
// sweep); next.wcount = popcount per word.
__global__ void k_union(GridGeom G, const uint64_t* __restrict__ kin, uint64_t* __restrict__ uout,
                        uint32_t* __restrict__ wcount)
{
    if (aborted(G.abort)) return;
    int64_t total = (int64_t)G.nb * G.RW;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
         i += (int64_t)gridDim.x * blockDim.x) {
        int64_t b = i / G.RW;
        int64_t rw = i - b * G.RW;
        int64_t row = rw / G.W;
        int w = (int)(rw - row * G.W);
        int y = (int)(row % G.n[1]);
        int z = (int)(row / G.n[1]);
        const uint64_t* seg = kin + b * G.RW;
        uint64_t acc = 0;
        for (int dz = -1; dz <= 1; dz++) {
            int zz = wrapi(z + dz, G.n[2]);
            for (int dy = -1; dy <= 1; dy++) {
                int yy = wrapi(y + dy, G.n[1]);
                const uint64_t* r = seg + ((int64_t)yy + (int64_t)G.n[1] * zz) * G.W;
                acc |= xdilate(r, G.W, G.n[0], w);
            }
        }
        acc &= word_mask(G.n[0], w);
        uout[i] = acc;
        wcount[i] = (uint32_t)__popcll(acc);
    }
}

__global__ void k_dense_u(const uint32_t* __restrict__ cnt, uint8_t* __restrict__ dense, int nb,
                          int64_t N, const int* abort)
{
    if (aborted(abort)) return;
    int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b < nb) dense[b] = (cnt[b] == (uint32_t)N) ? 1 : 0;
}

__global__ void k_dense_k(const uint32_t* __restrict__ kcnt, uint8_t* __restrict__ dense, int nb,
                          int64_t N, const int* abort, StepCounters* ctr)
{
    if (aborted(abort)) return;
    int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b < nb && kcnt[b] == (uint32_t)N) dense[b] |= 2;
    if (ctr && b == 0) ctr->done = 1;
}

// Capacity check of a step whose pools were sized before it ran (captured step
// sequences): when the union needs more slots than the pools hold, the step and every
// later one are skipped, leaving the last complete state in its layout.
__global__ void k_capacity(const int64_t* __restrict__ total, int64_t capacity, int* abort,
                           StepCounters* ctr)
{
    if (aborted(abort)) return;
    const int64_t t = *total;
    ctr->needed = (long long)t;
    if (t > capacity) {
        ctr->error |= 8;
        *abort = 1;
    }
}

constexpr int kPackThreads = 256;

// Sparsity rule: a slot of the new layout stays iff any of its four chunks had a value
// >= threshold (the per-chunk flags are written by the sweep epilogue).  Removed blocks
// add their FP64 mass (sum of the 64 averages) to the dropped mass.
template <int kCodec>
__global__ void k_pack_keep(GridGeom G, LayoutView L, const uint8_t* __restrict__ keepq,
                            uint64_t* __restrict__ kout, uint32_t* __restrict__ kcnt,
                            StepCounters* __restrict__ ctr, int64_t chunks_per_seg)
{
    if (aborted(G.abort)) return;
    __shared__ unsigned long long s_kept[kPackThreads / 32], s_drop[kPackThreads / 32];
    __shared__ double s_mass[kPackThreads / 32];
    const int64_t b = blockIdx.x / chunks_per_seg;
    const int64_t rw = (blockIdx.x % chunks_per_seg) * kPackThreads + threadIdx.x;
    unsigned long long kept = 0, drop = 0;
    double dmass = 0.0;
    if (rw < G.RW) {
        int64_t wi = b * G.RW + rw;
        uint64_t u = L.ubits[wi];
        uint64_t k = 0;
        uint32_t wo = L.woff[wi];
        int64_t bb = L.base[b];
        uint32_t cb = L.cnt[b];
        uint64_t rest = u;
        while (rest) {
            int bit = __ffsll((long long)rest) - 1;
            rest &= rest - 1;
            int64_t rank = (int64_t)wo + __popcll(u & ((1ull << bit) - 1ull));
            int64_t slot = bb + rank;
            uint32_t flags = *reinterpret_cast<const uint32_t*>(keepq + slot * 4);
            if (flags) {
                k |= 1ull << bit;
                kept++;
            } else {
                drop++;
                // the four chunks are loaded independently and each summed in FP32 (16
                // values of one block: relative error ~1e-7 of a dropped block's mass);
                // the chunk sums are accumulated in FP64
                using T = typename Codec<kCodec>::T;
                float cs[4];
#pragma unroll
                for (int q = 0; q < 4; q++) {
                    const int64_t ci = bb * 4 + (int64_t)q * cb + rank;  // chunk index
                    const float sc = kCodec ? L.scale[ci] : 1.0f;
                    const T* p = static_cast<const T*>(L.pool) + ci * kChunk;
                    float part[4] = {0.f, 0.f, 0.f, 0.f};
                    if constexpr (kCodec == 0) {
                        const float4* p4 = reinterpret_cast<const float4*>(p);
#pragma unroll
                        for (int j = 0; j < 4; j++) {
                            const float4 v = p4[j];
                            part[j] = (v.x + v.y) + (v.z + v.w);
                        }
                    } else {
#pragma unroll
                        for (int j = 0; j < kChunk; j++) part[j & 3] += Codec<kCodec>::dec(p[j], sc);
                    }
                    cs[q] = (part[0] + part[1]) + (part[2] + part[3]);
                }
                dmass += ((double)cs[0] + (double)cs[1]) + ((double)cs[2] + (double)cs[3]);
            }
        }
        kout[wi] = k;
    }
    // CTA reduction, one atomic per CTA
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int o = 16; o > 0; o >>= 1) {
        kept += __shfl_down_sync(0xffffffffu, kept, o);
        drop += __shfl_down_sync(0xffffffffu, drop, o);
        dmass += __shfl_down_sync(0xffffffffu, dmass, o);
    }
    if (lane == 0) {
        s_kept[warp] = kept;
        s_drop[warp] = drop;
        s_mass[warp] = dmass;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long K = 0, D = 0;
        double M = 0.0;
        for (int w = 0; w < kPackThreads / 32; w++) {
            K += s_kept[w];
            D += s_drop[w];
            M += s_mass[w];
        }
        if (K) atomicAdd(&kcnt[b], (uint32_t)K);
        if (K) atomicAdd(&ctr->kept, K);
        if (D) atomicAdd(&ctr->dropped, D);
        if (M != 0.0) atomicAdd(&ctr->dropped_mass, M);
    }
}

// ---- per-cell lists -> layout ----------------------------------------------------
__device__ __forceinline__ int64_t cell_of_block(const int64_t* off, int64_t N, int64_t t)
{
    int64_t lo = 0, hi = N;  // find c with off[c] <= t < off[c+1]
    while (hi - lo > 1) {
        int64_t mid = (lo + hi) >> 1;
        if (off[mid] <= t) lo = mid;
        else hi = mid;
    }
    return lo;
}

__global__ void k_check_offsets(const int64_t* __restrict__ off, int64_t N, int64_t M, int* err)
{
    int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c == 0 && (off[0] != 0 || off[N] != M)) atomicOr(err, 1);
    if (c < N && off[c + 1] < off[c]) atomicOr(err, 1);
}

__global__ void k_mark(GridGeom G, const int64_t* __restrict__ off, const uint16_t* __restrict__ ids,
                       int64_t M, uint64_t* __restrict__ ubits, int64_t* __restrict__ cell_of,
                       int* err)
{
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= M) return;
    int64_t c = cell_of_block(off, G.N, t);
    int b = ids[t];
    if (b >= G.nb) {
        atomicOr(err, 2);
        return;
    }
    if (t > off[c] && ids[t - 1] >= ids[t]) atomicOr(err, 4);
    cell_of[t] = c;
    int x = (int)(c % G.n[0]);
    int64_t row = c / G.n[0];
    atomicOr((unsigned long long*)&ubits[(int64_t)b * G.RW + row * G.W + (x >> 6)],
             (unsigned long long)(1ull << (x & 63)));
}

template <int kCodec>
__global__ void k_scatter(GridGeom G, LayoutView L, const uint16_t* __restrict__ ids,
                          const int64_t* __restrict__ cell_of, const float* __restrict__ vals,
                          int64_t t0, int64_t M)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= M * 64) return;
    int64_t t = t0 + (i >> 6);  // block index in the full list; vals holds blocks t0 ..
    int v = (int)(i & 63);
    int b = ids[t];
    int64_t c = cell_of[t];
    int x = (int)(c % G.n[0]);
    int64_t rank = cell_rank(L, G, b, x, c / G.n[0], false);
    int64_t dst = ((int64_t)L.base[b] * 4 + (int64_t)(v >> 4) * L.cnt[b] + rank) * kChunk + (v & 15);
    const float f = vals[i];
    float inv = 1.0f;
    if constexpr (kCodec != 0) {
        // the 16 values of a chunk are 16 consecutive threads (a half warp, since every
        // block's 64 values start at a warp boundary): their largest magnitude sets the
        // chunk's power-of-two scale
        const unsigned half = (threadIdx.x & 16) ? 0xffff0000u : 0x0000ffffu;
        const ChunkScale cs = chunk_scale(__uint_as_float(__reduce_max_sync(half, __float_as_uint(fabsf(f)))));
        if ((v & 15) == 0) L.scale[dst >> 4] = cs.s;
        inv = cs.inv;
    }
    static_cast<typename Codec<kCodec>::T*>(L.pool)[dst] = Codec<kCodec>::enc(f, inv);
}

// ---- layout -> per-cell lists ----------------------------------------------------
struct Window {
    int o[3], s[3];
    int64_t ncell;
};

// global (x, row) of window cell wc (x fastest), wrapping periodically
__device__ __forceinline__ void window_cell(const GridGeom& G, const Window& Wn, int64_t wc, int& x,
                                            int64_t& row)
{
    int wx = (int)(wc % Wn.s[0]);
    int64_t r = wc / Wn.s[0];
    int wy = (int)(r % Wn.s[1]);
    int wz = (int)(r / Wn.s[1]);
    x = wrapi(Wn.o[0] + wx, G.n[0]);
    int y = wrapi(Wn.o[1] + wy, G.n[1]);
    int z = wrapi(Wn.o[2] + wz, G.n[2]);
    row = y + (int64_t)G.n[1] * z;
}

__global__ void k_cell_counts(GridGeom G, Window Wn, const uint64_t* __restrict__ kbits,
                              uint32_t* __restrict__ cnt)
{
    int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= Wn.ncell) return;
    int x;
    int64_t row;
    window_cell(G, Wn, c, x, row);
    int64_t wo = row * G.W + (x >> 6);
    uint64_t bit = 1ull << (x & 63);
    uint32_t k = 0;
    for (int b = 0; b < G.nb; b++) k += (kbits[(int64_t)b * G.RW + wo] & bit) ? 1u : 0u;
    cnt[c] = k;
}

__global__ void k_offsets64(const uint32_t* __restrict__ excl, const int64_t* __restrict__ chunk_base,
                            int64_t chunk, int64_t N, int64_t* __restrict__ off)
{
    int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c < N) off[c] = chunk_base[c / chunk] + excl[c];
    if (c == 0) off[N] = chunk_base[(N + chunk - 1) / chunk];
}

__global__ void k_fill_ids(GridGeom G, Window Wn, LayoutView L, const int64_t* __restrict__ off,
                           uint16_t* __restrict__ ids, int64_t* __restrict__ rank_of)
{
    int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= Wn.ncell) return;
    int x;
    int64_t row;
    window_cell(G, Wn, c, x, row);
    int64_t wo = row * G.W + (x >> 6);
    uint64_t bit = 1ull << (x & 63);
    int64_t o = off[c];
    for (int b = 0; b < G.nb; b++) {
        if (L.kbits[(int64_t)b * G.RW + wo] & bit) {
            ids[o] = (uint16_t)b;
            rank_of[o] = cell_rank(L, G, b, x, row, false);
            o++;
        }
    }
}

template <int kCodec>
__global__ void k_gather(LayoutView L, const uint16_t* __restrict__ ids,
                         const int64_t* __restrict__ rank_of, float* __restrict__ vals, int64_t M)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= M * 64) return;
    int64_t t = i >> 6;
    int v = (int)(i & 63);
    int b = ids[t];
    const auto* pool = static_cast<const typename Codec<kCodec>::T*>(L.pool);
    const int64_t e = ((int64_t)L.base[b] * 4 + (int64_t)(v >> 4) * L.cnt[b] + rank_of[t]) * kChunk + (v & 15);
    vals[i] = Codec<kCodec>::dec(pool[e], kCodec ? L.scale[e >> 4] : 1.0f);
}

// ---- moments -----------------------------------------------------------------------
struct VMesh {
    double vmin[3], dv[3];
};

__device__ __forceinline__ double warp_sum(double x)
{
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    return x;
}

// One warp per cell; two passes over the cell's blocks (n and nV, then P about V).
template <int kCodec>
__global__ void k_moments(GridGeom G, LayoutView L, VMesh V, double* __restrict__ out)
{
    int64_t c = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    int lane = threadIdx.x & 31;
    if (c >= G.N) return;
    int x = (int)(c % G.n[0]);
    int64_t row = c / G.n[0];
    int64_t wo = row * G.W + (x >> 6);
    uint64_t bit = 1ull << (x & 63);
    double dv3 = V.dv[0] * V.dv[1] * V.dv[2];
    double s0 = 0, s1[3] = {0, 0, 0}, s2[3] = {0, 0, 0};
    double Vd[3] = {0, 0, 0};
    for (int pass = 0; pass < 2; pass++) {
        for (int b0 = 0; b0 < G.nb; b0 += 32) {
            int bl = b0 + lane;
            bool has = bl < G.nb && (L.kbits[(int64_t)bl * G.RW + wo] & bit);
            unsigned m = __ballot_sync(0xffffffffu, has);
            while (m) {
                int j = __ffs(m) - 1;
                m &= m - 1;
                int b = b0 + j;
                int64_t rank = cell_rank(L, G, b, x, row, false);
                int bx = b % G.nbx, by = (b / G.nbx) % G.nby, bz = b / (G.nbx * G.nby);
                for (int h = 0; h < 2; h++) {
                    int v = lane + 32 * h;
                    const auto* pool = static_cast<const typename Codec<kCodec>::T*>(L.pool);
                    const int64_t e =
                        ((int64_t)L.base[b] * 4 + (int64_t)(v >> 4) * L.cnt[b] + rank) * kChunk + (v & 15);
                    float f = Codec<kCodec>::dec(pool[e], kCodec ? L.scale[e >> 4] : 1.0f);
                    double vel[3] = {V.vmin[0] + (bx * 4 + (v & 3) + 0.5) * V.dv[0],
                                     V.vmin[1] + (by * 4 + ((v >> 2) & 3) + 0.5) * V.dv[1],
                                     V.vmin[2] + (bz * 4 + (v >> 4) + 0.5) * V.dv[2]};
                    if (pass == 0) {
                        s0 += f;
                        for (int d = 0; d < 3; d++) s1[d] += vel[d] * f;
                    } else {
                        for (int d = 0; d < 3; d++) s2[d] += (vel[d] - Vd[d]) * (vel[d] - Vd[d]) * f;
                    }
                }
            }
        }
        if (pass == 0) {
            s0 = warp_sum(s0);
            for (int d = 0; d < 3; d++) s1[d] = warp_sum(s1[d]);
            for (int d = 0; d < 3; d++) Vd[d] = s0 != 0.0 ? s1[d] / s0 : 0.0;
        }
    }
    for (int d = 0; d < 3; d++) s2[d] = warp_sum(s2[d]);
    if (lane == 0) {
        double* o = out + c * 7;
        o[0] = s0 * dv3;
        for (int d = 0; d < 3; d++) o[1 + d] = s1[d] * dv3;
        for (int d = 0; d < 3; d++) o[4 + d] = s2[d] * dv3;
    }
}

__global__ void k_fill_f32(float* __restrict__ p, float v, int64_t n)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) p[i] = v;
}


__global__ void k_popcount(const uint64_t* __restrict__ u, uint32_t* __restrict__ c, int64_t n)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) c[i] = (uint32_t)__popcll(u[i]);
}

__global__ void k_sum_density(const double* __restrict__ mom, int64_t N, double* __restrict__ out)
{
    double s = 0.0;
    for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < N;
         c += (int64_t)gridDim.x * blockDim.x)
        s += mom[c * 7];
    s = warp_sum(s);
    if ((threadIdx.x & 31) == 0) atomicAdd(out, s);
}

inline int nblk(int64_t n, int t) { return (int)((n + t - 1) / t); }

}  // namespace

// ---------------------------------------------------------------------------------
void launch_seg_scan(const uint32_t* in, uint32_t* out, uint32_t* seg_total, int64_t seg_len,
                     int64_t nseg, cudaStream_t s, const int* abort)
{
    if (nseg <= 0) return;
    int threads = seg_len >= 1024 ? kScanThreads : (seg_len >= 256 ? 256 : 64);
    k_seg_scan<<<(unsigned)nseg, threads, 0, s>>>(in, out, seg_total, seg_len, abort); note_launch();
}

void launch_base_scan(const uint32_t* seg_total, int64_t* base, int64_t nseg, cudaStream_t s,
                      const int* abort)
{
    k_base_scan<<<1, kScanThreads, 0, s>>>(seg_total, base, nseg, abort); note_launch();
}

void launch_capacity_check(Grid* g, const Layout& L, int64_t capacity, StepCounters* ctr)
{
    k_capacity<<<1, 1, 0, g->stream>>>(L.base + g->geom.nb, capacity, g->abort_flag, ctr);
    note_launch();
}

vl_status layout_alloc_meta(Grid* g, Layout& L)
{
    const GridGeom& G = g->geom;
    size_t words = (size_t)G.nb * (size_t)G.RW;
    L.ubits = (uint64_t*)g->alloc(words * 8);
    L.kbits = (uint64_t*)g->alloc(words * 8);
    L.woff = (uint32_t*)g->alloc(words * 4);
    L.wcount = (uint32_t*)g->alloc(words * 4);
    L.cnt = (uint32_t*)g->alloc((size_t)G.nb * 4);
    L.base = (int64_t*)g->alloc(((size_t)G.nb + 1) * 8);
    L.dense = (uint8_t*)g->alloc((size_t)G.nb);
    L.kcnt = (uint32_t*)g->alloc((size_t)G.nb * 4);
    if (!L.ubits || !L.kbits || !L.woff || !L.wcount || !L.cnt || !L.base || !L.dense || !L.kcnt)
        return fail(g, VL_ENOMEM, "allocation of the block bitmaps failed");
    cudaMemsetAsync(L.ubits, 0, words * 8, g->stream);
    cudaMemsetAsync(L.kbits, 0, words * 8, g->stream);
    cudaMemsetAsync(L.dense, 0, (size_t)G.nb, g->stream);
    return VL_OK;
}

void layout_free(Grid* g, Layout& L)
{
    g->release(L.ubits);
    g->release(L.kbits);
    g->release(L.woff);
    g->release(L.wcount);
    g->release(L.cnt);
    g->release(L.base);
    g->release(L.dense);
    g->release(L.kcnt);
    g->release(L.scale);
    g->release(L.pool);
    g->release(L.keepq);
    L = Layout{};
}

void layout_release_pool(Grid* g, Layout& L)
{
    cudaStreamSynchronize(g->stream);  // no queued kernel may still use the pool
    g->release(L.pool);
    g->release(L.keepq);
    g->release(L.scale);
    L.pool = nullptr;
    L.keepq = nullptr;
    L.scale = nullptr;
    L.capacity = 0;
}

vl_status layout_ensure_pool(Grid* g, Layout& L, int64_t blocks)
{
    if (blocks <= L.capacity && L.pool) return VL_OK;
    int64_t cap = blocks + blocks / 32 + 64;
    g->release(L.pool);
    g->release(L.keepq);
    g->release(L.scale);
    L.pool = g->alloc((size_t)cap * 64 * g->esize);
    L.keepq = (uint8_t*)g->alloc((size_t)cap * 4);
    // 16-bit storage: one power-of-two scale per chunk of 16 values
    L.scale = g->codec ? (float*)g->alloc((size_t)cap * 4 * sizeof(float)) : nullptr;
    if (!L.pool || !L.keepq || (g->codec && !L.scale)) {
        L.capacity = 0;
        return fail(g, VL_ENOMEM, "allocation of the phase-space pool failed (" +
                                      std::to_string(cap * 64 * (int64_t)g->esize) + " bytes)");
    }
    L.capacity = cap;
    return VL_OK;
}

void launch_index(Grid* g, Layout& L)
{
    const GridGeom& G = g->geom;
    launch_seg_scan(L.wcount, L.woff, L.cnt, G.RW, G.nb, g->stream, G.abort);
    launch_base_scan(L.cnt, L.base, G.nb, g->stream, G.abort);
    k_dense_u<<<nblk(G.nb, 256), 256, 0, g->stream>>>(L.cnt, L.dense, G.nb, G.N, G.abort); note_launch();
}

vl_status layout_grow_pool(Grid* g, Layout& L, int64_t blocks)
{
    if (blocks <= L.capacity && L.pool) return VL_OK;
    void* pool = g->alloc((size_t)blocks * 64 * g->esize);
    uint8_t* keepq = (uint8_t*)g->alloc((size_t)blocks * 4);
    float* scale = g->codec ? (float*)g->alloc((size_t)blocks * 4 * sizeof(float)) : nullptr;
    if (!pool || !keepq || (g->codec && !scale)) {
        g->release(pool);
        g->release(keepq);
        g->release(scale);
        return fail(g, VL_ENOMEM, "growing the phase-space pool failed (" + std::to_string(blocks * 64 * (int64_t)g->esize) + " bytes)");
    }
    if (L.pool && L.total > 0) {
        const int64_t kept = std::min(L.total, L.capacity);
        cudaMemcpyAsync(pool, L.pool, (size_t)kept * 64 * g->esize, cudaMemcpyDeviceToDevice, g->stream);
        if (scale && L.scale)
            cudaMemcpyAsync(scale, L.scale, (size_t)kept * 4 * sizeof(float), cudaMemcpyDeviceToDevice, g->stream);
    }
    cudaStreamSynchronize(g->stream);
    g->release(L.pool);
    g->release(L.keepq);
    g->release(L.scale);
    L.pool = pool;
    L.keepq = keepq;
    L.scale = scale;
    L.capacity = blocks;
    return VL_OK;
}

vl_status layout_index(Grid* g, Layout& L, int64_t* total)
{
    const GridGeom& G = g->geom;
    launch_index(g, L);
    cudaMemcpyAsync(g->host_scalar, L.base + G.nb, 8, cudaMemcpyDeviceToHost, g->stream);
    cudaError_t e = cudaStreamSynchronize(g->stream);
    if (e != cudaSuccess) return cuda_fail(g, e, "layout index");
    *total = g->host_scalar[0];
    L.total = *total;
    return VL_OK;
}

void launch_union(Grid* g, const Layout& cur, Layout& next)
{
    const GridGeom& G = g->geom;
    int64_t total = (int64_t)G.nb * G.RW;
    int blocks = (int)std::min<int64_t>(nblk(total, 256), 152 * 32);
    k_union<<<blocks, 256, 0, g->stream>>>(G, cur.kbits, next.ubits, next.wcount); note_launch();
}

void launch_pack_keep(Grid* g, Layout& next, StepCounters* ctr)
{
    const GridGeom& G = g->geom;
    int64_t cps = (G.RW + kPackThreads - 1) / kPackThreads;
    cudaMemsetAsync(next.kcnt, 0, (size_t)G.nb * 4, g->stream);
    with_codec(g->codec, [&](auto c) {
        k_pack_keep<decltype(c)::value><<<(unsigned)(cps * G.nb), kPackThreads, 0, g->stream>>>(
            G, next.view(), next.keepq, next.kbits, next.kcnt, ctr, cps);
    });
    note_launch();
    k_dense_k<<<nblk(G.nb, 256), 256, 0, g->stream>>>(next.kcnt, next.dense, G.nb, G.N, G.abort, ctr);
    note_launch();
}


namespace {
struct Scratch {
    Grid* g;
    std::vector<void*> ptrs;
    explicit Scratch(Grid* gg) : g(gg) {}
    void* get(size_t bytes)
    {
        void* p = g->alloc(bytes);
        if (p) ptrs.push_back(p);
        return p;
    }
    ~Scratch()
    {
        // frees are stream-ordered for the caching allocator; synchronise first so that
        // no kernel still reads a buffer handed back to cudaFree-based allocators
        cudaStreamSynchronize(g->stream);
        for (void* p : ptrs) g->release(p);
    }
};
}  // namespace

// Device address of a page-locked host buffer (cudaHostAlloc, cudaMallocHost or
// cudaHostRegister), through which kernels read and write it directly -- over
// NVLink-C2C on a Grace host -- or nullptr for any other pointer.
static void* mapped_host(const void* p)
{
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return a.type == cudaMemoryTypeHost ? a.devicePointer : nullptr;
}

vl_status set_blocks(Grid* g, int64_t M, const int64_t* off_in, const uint16_t* ids_in,
                     const float* vals_in, int on_device)
{
    const GridGeom& G = g->geom;
    cudaStream_t s = g->stream;
    if (M < 0 || !off_in || (M > 0 && (!ids_in || !vals_in)))
        return fail(g, VL_EINVAL, "vl_set_blocks: null pointer or negative block count");
    Scratch sc(g);
    const int64_t* off = off_in;
    const uint16_t* ids = ids_in;
    // host values: read in place by the scatter kernel when the buffer is page-locked,
    // else streamed through device staging buffers below
    const float* mapped = (!on_device && M > 0) ? static_cast<const float*>(mapped_host(vals_in)) : nullptr;
    const float* vals = on_device ? vals_in : mapped;
    if (!on_device) {
        int64_t* d_off = (int64_t*)sc.get((size_t)(G.N + 1) * 8);
        uint16_t* d_ids = (uint16_t*)sc.get((size_t)std::max<int64_t>(M, 1) * 2);
        if (!d_off || !d_ids) return fail(g, VL_ENOMEM, "vl_set_blocks: staging allocation failed");
        cudaMemcpyAsync(d_off, off_in, (size_t)(G.N + 1) * 8, cudaMemcpyHostToDevice, s);
        if (M > 0) cudaMemcpyAsync(d_ids, ids_in, (size_t)M * 2, cudaMemcpyHostToDevice, s);
        off = d_off;
        ids = d_ids;
    }
    Layout& L = g->lay[g->cur];
    size_t words = (size_t)G.nb * (size_t)G.RW;
    int64_t* cell_of = (int64_t*)sc.get((size_t)std::max<int64_t>(M, 1) * 8);
    int* err = (int*)sc.get(sizeof(int));
    if (!cell_of || !err) return fail(g, VL_ENOMEM, "vl_set_blocks: scratch allocation failed");
    cudaMemsetAsync(err, 0, sizeof(int), s);
    cudaMemsetAsync(L.ubits, 0, words * 8, s);
    k_check_offsets<<<nblk(G.N + 1, 256), 256, 0, s>>>(off, G.N, M, err); note_launch();
    if (M > 0) { k_mark<<<nblk(M, 256), 256, 0, s>>>(G, off, ids, M, L.ubits, cell_of, err); note_launch(); }
    cudaMemcpyAsync(g->host_scalar, err, sizeof(int), cudaMemcpyDeviceToHost, s);
    cudaError_t e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(g, e, "vl_set_blocks");
    int herr = (int)(g->host_scalar[0] & 0xffffffff);
    if (herr & 1) return fail(g, VL_EINVAL, "vl_set_blocks: cell offsets must start at 0, be non-decreasing and end at nblocks");
    if (herr & 2) return fail(g, VL_EINVAL, "vl_set_blocks: block id out of range of the velocity mesh");
    if (herr & 4) return fail(g, VL_EINVAL, "vl_set_blocks: block ids must be strictly increasing within a cell");
    k_popcount<<<nblk((int64_t)words, 256), 256, 0, s>>>(L.ubits, L.wcount, (int64_t)words); note_launch();
    cudaMemcpyAsync(L.kbits, L.ubits, words * 8, cudaMemcpyDeviceToDevice, s);
    int64_t total = 0;
    vl_status st = layout_index(g, L, &total);
    if (st != VL_OK) return st;
    if (total != M) return fail(g, VL_EINVAL, "vl_set_blocks: duplicate block ids");
    k_dense_k<<<nblk(G.nb, 256), 256, 0, s>>>(L.cnt, L.dense, G.nb, G.N, nullptr, nullptr); note_launch();
    st = layout_ensure_pool(g, L, std::max<int64_t>(M, 1));
    if (st != VL_OK) return st;
    const int64_t chunk = std::min<int64_t>(std::max<int64_t>(M, 1), (int64_t)1 << 22);  // 1 GiB of values
    // host values: copied in chunks (the device never holds a second full copy) through
    // two staging buffers on a copy stream, so that the copy of one chunk overlaps the
    // kernel that consumes the previous one
    float* stage_buf[2] = {nullptr, nullptr};
    cudaEvent_t ready = nullptr, copied[2] = {nullptr, nullptr}, used[2] = {nullptr, nullptr};
    const bool staged = M > 0 && !on_device && !mapped;
    const bool direct = on_device || mapped;  // the kernels read vals in place
    // two buffers when more than one chunk goes through them
    const int nbuf = ((M + chunk - 1) / chunk > 1) ? 2 : 1;
    if (staged) {
        for (int i = 0; i < nbuf; i++) {
            stage_buf[i] = (float*)sc.get((size_t)chunk * 256);
            if (!stage_buf[i]) return fail(g, VL_ENOMEM, "vl_set_blocks: staging allocation failed");
        }
        if (!g->copy_stream) {
            e = cudaStreamCreateWithFlags(&g->copy_stream, cudaStreamNonBlocking);
            if (e != cudaSuccess) return cuda_fail(g, e, "vl_set_blocks: copy stream");
        }
        cudaEventCreateWithFlags(&ready, cudaEventDisableTiming);
        for (int i = 0; i < 2; i++) {
            cudaEventCreateWithFlags(&copied[i], cudaEventDisableTiming);
            cudaEventCreateWithFlags(&used[i], cudaEventDisableTiming);
        }
        cudaEventRecord(ready, s);  // the staging buffers are free for the copy stream
        cudaStreamWaitEvent(g->copy_stream, ready, 0);
    }
    int64_t k = 0;  // chunk counter (staging buffer k % nbuf)
    for (int64_t t0 = 0; t0 < M; t0 += (direct ? M : chunk), k++) {
        const int64_t m = direct ? M : std::min(chunk, M - t0);
        const int bi = (int)(k % nbuf);
        const float* v = direct ? vals : stage_buf[bi];
        if (staged) {
            if (k >= nbuf) cudaStreamWaitEvent(g->copy_stream, used[bi], 0);  // chunk k-nbuf consumed
            cudaMemcpyAsync(stage_buf[bi], vals_in + t0 * 64, (size_t)m * 256, cudaMemcpyHostToDevice,
                            g->copy_stream);
            cudaEventRecord(copied[bi], g->copy_stream);
            cudaStreamWaitEvent(s, copied[bi], 0);
        }
        with_codec(g->codec, [&](auto c) {
            k_scatter<decltype(c)::value><<<nblk(m * 64, 256), 256, 0, s>>>(G, L.view(), ids, cell_of, v, t0, m);
        });
        note_launch();
        if (staged) cudaEventRecord(used[bi], s);
    }
    if (staged) {
        cudaStreamSynchronize(s);  // every copy was waited for by a kernel on s
        cudaEventDestroy(ready);
        for (int i = 0; i < 2; i++) {
            cudaEventDestroy(copied[i]);
            cudaEventDestroy(used[i]);
        }
    }
    e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(g, e, "vl_set_blocks scatter");
    g->has_state = true;
    return VL_OK;
}

namespace {
Window make_window(const GridGeom& G, const int* origin, const int* size)
{
    Window Wn;
    Wn.ncell = 1;
    for (int d = 0; d < 3; d++) {
        Wn.o[d] = origin ? origin[d] : 0;
        Wn.s[d] = size ? size[d] : G.n[d];
        Wn.ncell *= Wn.s[d];
    }
    return Wn;
}
}  // namespace

// Per-cell lists of a box window of the grid (the whole grid when origin/size are
// NULL).  With count_only, only *count is produced.
vl_status get_window(Grid* g, const int* origin, const int* size, int64_t capacity,
                     int64_t* off_out, uint16_t* ids_out, float* vals_out, int on_device,
                     int64_t* count)
{
    const GridGeom& G = g->geom;
    const Layout& L = g->lay[g->cur];
    cudaStream_t s = g->stream;
    if (size)
        for (int d = 0; d < 3; d++)
            if (size[d] <= 0 || size[d] > G.n[d])
                return fail(g, VL_EINVAL, "window size must be within 1..n per dimension");
    Window Wn = make_window(G, origin, size);
    Scratch sc(g);
    const int64_t chunk = 4096;
    int64_t nchunk = (Wn.ncell + chunk - 1) / chunk;
    uint32_t* ccnt = (uint32_t*)sc.get((size_t)nchunk * chunk * 4);
    uint32_t* cexc = (uint32_t*)sc.get((size_t)nchunk * chunk * 4);
    uint32_t* ctot = (uint32_t*)sc.get((size_t)nchunk * 4);
    int64_t* cbase = (int64_t*)sc.get(((size_t)nchunk + 1) * 8);
    if (!ccnt || !cexc || !ctot || !cbase) return fail(g, VL_ENOMEM, "block listing: scratch allocation failed");
    cudaMemsetAsync(ccnt, 0, (size_t)nchunk * chunk * 4, s);
    k_cell_counts<<<nblk(Wn.ncell, 256), 256, 0, s>>>(G, Wn, L.kbits, ccnt); note_launch();
    launch_seg_scan(ccnt, cexc, ctot, chunk, nchunk, s, nullptr);
    launch_base_scan(ctot, cbase, nchunk, s, nullptr);
    cudaMemcpyAsync(g->host_scalar, cbase + nchunk, 8, cudaMemcpyDeviceToHost, s);
    cudaError_t e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(g, e, "block listing");
    const int64_t M = g->host_scalar[0];
    if (count) *count = M;
    if (!off_out) return VL_OK;
    if (capacity < M)
        return fail(g, VL_ECAPACITY, "vl_get_blocks: capacity " + std::to_string(capacity) +
                                         " < " + std::to_string(M) + " blocks");
    if (M > 0 && (!ids_out || !vals_out)) return fail(g, VL_EINVAL, "vl_get_blocks: null pointer");
    int64_t* rank_of = (int64_t*)sc.get((size_t)std::max<int64_t>(M, 1) * 8);
    int64_t* d_off = on_device ? off_out : (int64_t*)sc.get((size_t)(Wn.ncell + 1) * 8);
    uint16_t* d_ids = on_device ? ids_out : (uint16_t*)sc.get((size_t)std::max<int64_t>(M, 1) * 2);
    // values into a page-locked host buffer: the gather kernel writes them in place
    float* mapped = (!on_device && M > 0) ? static_cast<float*>(mapped_host(vals_out)) : nullptr;
    float* d_vals = on_device ? vals_out : (mapped ? mapped : (float*)sc.get((size_t)std::max<int64_t>(M, 1) * 256));
    if (!rank_of || !d_off || !d_ids || !d_vals) return fail(g, VL_ENOMEM, "vl_get_blocks: scratch allocation failed");
    k_offsets64<<<nblk(Wn.ncell + 1, 256), 256, 0, s>>>(cexc, cbase, chunk, Wn.ncell, d_off); note_launch();
    k_fill_ids<<<nblk(Wn.ncell, 128), 128, 0, s>>>(G, Wn, L.view(), d_off, d_ids, rank_of); note_launch();
    if (M > 0) {
        with_codec(g->codec, [&](auto c) {
            k_gather<decltype(c)::value><<<nblk(M * 64, 256), 256, 0, s>>>(L.view(), d_ids, rank_of, d_vals, M);
        });
        note_launch();
    }
    if (!on_device) {
        cudaMemcpyAsync(off_out, d_off, (size_t)(Wn.ncell + 1) * 8, cudaMemcpyDeviceToHost, s);
        if (M > 0) {
            cudaMemcpyAsync(ids_out, d_ids, (size_t)M * 2, cudaMemcpyDeviceToHost, s);
            if (!mapped) cudaMemcpyAsync(vals_out, d_vals, (size_t)M * 256, cudaMemcpyDeviceToHost, s);
        }
    }
    e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(g, e, "vl_get_blocks");
    return VL_OK;
}

vl_status get_block_count(Grid* g, int64_t* n)
{
    return get_window(g, nullptr, nullptr, 0, nullptr, nullptr, nullptr, 0, n);
}

vl_status get_blocks(Grid* g, int64_t capacity, int64_t* off_out, uint16_t* ids_out,
                     float* vals_out, int on_device)
{
    if (!off_out || capacity < 0) return fail(g, VL_EINVAL, "vl_get_blocks: null pointer");
    return get_window(g, nullptr, nullptr, capacity, off_out, ids_out, vals_out, on_device, nullptr);
}

namespace {
// Window block t -> its cell in the grid (planes from z0, wrapping); err |= 1 when the
// cell does not hold that block id in the current layout, 2 when the id is out of range.
__global__ void k_window_cells(GridGeom G, LayoutView L, const int64_t* __restrict__ off_w, int64_t nw,
                               const uint16_t* __restrict__ ids_w, int64_t Mw, int z0,
                               int64_t* __restrict__ cell_of, int* err)
{
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= Mw) return;
    const int64_t wc = cell_of_block(off_w, nw, t);
    const int64_t nxy = (int64_t)G.n[0] * G.n[1];
    const int64_t c = wc % nxy + (int64_t)wrapi(z0 + (int)(wc / nxy), G.n[2]) * nxy;
    const int b = ids_w[t];
    if (b >= G.nb) {
        atomicOr(err, 2);
        return;
    }
    cell_of[t] = c;
    const int x = (int)(c % G.n[0]);
    const int64_t wi = (int64_t)b * G.RW + (c / G.n[0]) * G.W + (x >> 6);
    if (!((L.kbits[wi] >> (x & 63)) & 1ull)) atomicOr(err, 1);
}

// dst_off[d0 + i] = src_off[s0 + i] - src_off[s0] + base, i = 0 .. n-1
__global__ void k_shift_offsets(const int64_t* __restrict__ src_off, int64_t s0, int64_t n, int64_t base,
                                int64_t* __restrict__ dst_off, int64_t d0)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) dst_off[d0 + i] = src_off[s0 + i] - src_off[s0] + base;
}
}  // namespace

// Replaces the blocks of z-planes z0 .. z0+nplanes-1 (wrapping) by the window lists and
// keeps every other cell.  A set of whole z-planes is one or two contiguous ranges of
// the cell order (x fastest, then y, then z), so the new lists are runs of the old and
// the window lists joined end to end: device copies of ids and values, shifted offsets,
// then the layout rebuilt from the joined lists by set_blocks.
vl_status set_blocks_planes(Grid* g, int z0, int nplanes, int64_t Mw, const int64_t* off_w_in,
                            const uint16_t* ids_w_in, const float* vals_w_in, int on_device)
{
    const GridGeom& G = g->geom;
    cudaStream_t s = g->stream;
    if (!g->has_state) return fail(g, VL_ESTATE, "vl_set_blocks_planes: no state (call vl_set_blocks first)");
    if (nplanes < 1 || nplanes > G.n[2] || Mw < 0 || !off_w_in || (Mw > 0 && (!ids_w_in || !vals_w_in)))
        return fail(g, VL_EINVAL, "vl_set_blocks_planes: 1 <= nplanes <= nz, lists required");
    const int64_t nxy = (int64_t)G.n[0] * G.n[1];
    const int64_t nw = nxy * nplanes;
    Scratch sc(g);
    // the window lists on the device
    const int64_t* off_w = off_w_in;
    const uint16_t* ids_w = ids_w_in;
    const float* vals_w = vals_w_in;
    if (!on_device) {
        int64_t* a = (int64_t*)sc.get((size_t)(nw + 1) * 8);
        uint16_t* b = (uint16_t*)sc.get((size_t)std::max<int64_t>(Mw, 1) * 2);
        float* c = (float*)sc.get((size_t)std::max<int64_t>(Mw, 1) * 256);
        if (!a || !b || !c) return fail(g, VL_ENOMEM, "vl_set_blocks_planes: staging allocation failed");
        cudaMemcpyAsync(a, off_w_in, (size_t)(nw + 1) * 8, cudaMemcpyHostToDevice, s);
        if (Mw > 0) {
            cudaMemcpyAsync(b, ids_w_in, (size_t)Mw * 2, cudaMemcpyHostToDevice, s);
            cudaMemcpyAsync(c, vals_w_in, (size_t)Mw * 256, cudaMemcpyHostToDevice, s);
        }
        off_w = a;
        ids_w = b;
        vals_w = c;
    }
    // fast path: the window keeps its block set (every listed block is present and the
    // window holds as many), so the values go into their slots in place (16-bit storage:
    // with the chunk scales of the new values)
    {
        const int origin[3] = {0, 0, z0};
        const int size[3] = {G.n[0], G.n[1], nplanes};
        int64_t Mcur = -1;
        vl_status st0 = get_window(g, origin, size, 0, nullptr, nullptr, nullptr, 0, &Mcur);
        if (st0 != VL_OK) return st0;
        if (Mcur == Mw) {
            int64_t* cell_of = (int64_t*)sc.get((size_t)std::max<int64_t>(Mw, 1) * 8);
            int* err = (int*)sc.get(sizeof(int));
            if (!cell_of || !err) return fail(g, VL_ENOMEM, "vl_set_blocks_planes: scratch allocation failed");
            Layout& L = g->lay[g->cur];
            cudaMemsetAsync(err, 0, sizeof(int), s);
            if (Mw > 0) {
                k_window_cells<<<nblk(Mw, 256), 256, 0, s>>>(G, L.view(), off_w, nw, ids_w, Mw, z0, cell_of, err);
                note_launch();
            }
            cudaMemcpyAsync(g->host_scalar, err, sizeof(int), cudaMemcpyDeviceToHost, s);
            cudaError_t e = cudaStreamSynchronize(s);
            if (e != cudaSuccess) return cuda_fail(g, e, "vl_set_blocks_planes");
            const int herr = (int)(g->host_scalar[0] & 0xffffffff);
            if (herr & 2) return fail(g, VL_EINVAL, "vl_set_blocks_planes: block id out of range of the velocity mesh");
            if (herr == 0) {
                if (Mw > 0) {
                    with_codec(g->codec, [&](auto c) {
                        k_scatter<decltype(c)::value>
                            <<<nblk(Mw * 64, 256), 256, 0, s>>>(G, L.view(), ids_w, cell_of, vals_w, 0, Mw);
                    });
                    note_launch();
                }
                e = cudaStreamSynchronize(s);
                return e == cudaSuccess ? VL_OK : cuda_fail(g, e, "vl_set_blocks_planes");
            }
        }
    }
    // the whole current state as lists on the device
    int64_t Mo = 0;
    vl_status st = get_window(g, nullptr, nullptr, 0, nullptr, nullptr, nullptr, 0, &Mo);
    if (st != VL_OK) return st;
    int64_t* off_o = (int64_t*)sc.get((size_t)(G.N + 1) * 8);
    uint16_t* ids_o = (uint16_t*)sc.get((size_t)std::max<int64_t>(Mo, 1) * 2);
    float* vals_o = (float*)sc.get((size_t)std::max<int64_t>(Mo, 1) * 256);
    if (!off_o || !ids_o || !vals_o) return fail(g, VL_ENOMEM, "vl_set_blocks_planes: scratch allocation failed");
    st = get_window(g, nullptr, nullptr, Mo, off_o, ids_o, vals_o, 1, nullptr);
    if (st != VL_OK) return st;
    // runs in the new cell order: (source lists, first source cell, cells)
    struct Run {
        int kind;  // 0: old state, 1: window lists
        int64_t s0, n;
    };
    const int64_t c0 = (int64_t)(((z0 % G.n[2]) + G.n[2]) % G.n[2]) * nxy;
    const int64_t lenA = std::min(nw, G.N - c0);  // window cells before the wrap
    std::vector<Run> runs;
    if (lenA == nw) {
        if (c0 > 0) runs.push_back({0, 0, c0});
        runs.push_back({1, 0, nw});
        if (c0 + nw < G.N) runs.push_back({0, c0 + nw, G.N - c0 - nw});
    } else {
        const int64_t cb = nw - lenA;  // window cells after the wrap, at cells 0 .. cb-1
        runs.push_back({1, lenA, cb});
        if (c0 > cb) runs.push_back({0, cb, c0 - cb});
        runs.push_back({1, 0, lenA});
    }
    // block ranges of the runs (host copies of the offsets at the run bounds)
    std::vector<int64_t> lo(runs.size()), hi(runs.size());
    for (size_t i = 0; i < runs.size(); i++) {
        const int64_t* off = runs[i].kind ? off_w : off_o;
        cudaMemcpyAsync(&g->host_scalar[0], off + runs[i].s0, 8, cudaMemcpyDeviceToHost, s);
        cudaMemcpyAsync(&g->host_scalar[1], off + runs[i].s0 + runs[i].n, 8, cudaMemcpyDeviceToHost, s);
        cudaError_t e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return cuda_fail(g, e, "vl_set_blocks_planes");
        lo[i] = g->host_scalar[0];
        hi[i] = g->host_scalar[1];
        if (hi[i] < lo[i]) return fail(g, VL_EINVAL, "vl_set_blocks_planes: cell offsets must be non-decreasing");
    }
    int64_t M = 0;
    for (size_t i = 0; i < runs.size(); i++) M += hi[i] - lo[i];
    int64_t* off_n = (int64_t*)sc.get((size_t)(G.N + 1) * 8);
    uint16_t* ids_n = (uint16_t*)sc.get((size_t)std::max<int64_t>(M, 1) * 2);
    float* vals_n = (float*)sc.get((size_t)std::max<int64_t>(M, 1) * 256);
    if (!off_n || !ids_n || !vals_n) return fail(g, VL_ENOMEM, "vl_set_blocks_planes: scratch allocation failed");
    int64_t d0 = 0, base = 0;
    for (size_t i = 0; i < runs.size(); i++) {
        const bool w = runs[i].kind != 0;
        const int64_t nb = hi[i] - lo[i];
        k_shift_offsets<<<nblk(runs[i].n, 256), 256, 0, s>>>(w ? off_w : off_o, runs[i].s0, runs[i].n, base, off_n, d0);
        note_launch();
        if (nb > 0) {
            cudaMemcpyAsync(ids_n + base, (w ? ids_w : ids_o) + lo[i], (size_t)nb * 2, cudaMemcpyDeviceToDevice, s);
            cudaMemcpyAsync(vals_n + base * 64, (w ? vals_w : vals_o) + lo[i] * 64, (size_t)nb * 256,
                            cudaMemcpyDeviceToDevice, s);
        }
        d0 += runs[i].n;
        base += nb;
    }
    g->host_scalar[0] = M;
    cudaMemcpyAsync(off_n + G.N, &g->host_scalar[0], 8, cudaMemcpyHostToDevice, s);
    cudaError_t e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(g, e, "vl_set_blocks_planes");
    return set_blocks(g, M, off_n, ids_n, vals_n, 1);
}

vl_status moments(Grid* g, double* out, int on_device)
{
    const GridGeom& G = g->geom;
    const Layout& L = g->lay[g->cur];
    if (!out) return fail(g, VL_EINVAL, "vl_moments: null pointer");
    Scratch sc(g);
    double* d_out = on_device ? out : (double*)sc.get((size_t)G.N * 7 * 8);
    if (!d_out) return fail(g, VL_ENOMEM, "vl_moments: scratch allocation failed");
    VMesh V;
    for (int d = 0; d < 3; d++) {
        V.vmin[d] = g->vmesh.vmin[d];
        V.dv[d] = g->vmesh.dv[d];
    }
    with_codec(g->codec, [&](auto c) {
        k_moments<decltype(c)::value><<<nblk(G.N * 32, 256), 256, 0, g->stream>>>(G, L.view(), V, d_out);
    });
    note_launch();
    if (!on_device)
        cudaMemcpyAsync(out, d_out, (size_t)G.N * 7 * 8, cudaMemcpyDeviceToHost, g->stream);
    cudaError_t e = cudaStreamSynchronize(g->stream);
    if (e != cudaSuccess) return cuda_fail(g, e, "vl_moments");
    return VL_OK;
}

vl_status total_mass(Grid* g, double* mass)
{
    const GridGeom& G = g->geom;
    Scratch sc(g);
    double* mom = (double*)sc.get((size_t)G.N * 7 * 8);
    double* acc = (double*)sc.get(8);
    if (!mom || !acc) return fail(g, VL_ENOMEM, "vl_mass: scratch allocation failed");
    vl_status st = moments(g, mom, 1);
    if (st != VL_OK) return st;
    cudaMemsetAsync(acc, 0, 8, g->stream);
    k_sum_density<<<152 * 4, 256, 0, g->stream>>>(mom, G.N, acc); note_launch();
    double h = 0.0;
    cudaMemcpyAsync(&h, acc, 8, cudaMemcpyDeviceToHost, g->stream);
    cudaError_t e = cudaStreamSynchronize(g->stream);
    if (e != cudaSuccess) return cuda_fail(g, e, "vl_mass");
    *mass = h * g->space.dx[0] * g->space.dx[1] * g->space.dx[2];
    return VL_OK;
}

}  // namespace vlgt
