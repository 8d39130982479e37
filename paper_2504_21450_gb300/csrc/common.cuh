// common.cuh -- data layout and device helpers shared by the CUDA kernels of libvlgt.
//
// Phase-space layout in HBM (one "layout" = one state of the sparse velocity space):
//   * For every block id b, a bitmap over the spatial cells, row by row: row = y + ny*z,
//     W = ceil(nx/64) 64-bit words per row, bit x%64 of word x/64.
//       ubits[b][row*W + w]  a slot exists for (cell, b) in this layout
//       kbits[b][row*W + w]  the block is present (kept); always a subset of ubits
//     The rank of a cell among the set ubits bits of segment b is its slot:
//       rank = woff[b][row*W + w] + popc(ubits word & bits below x)
//     (a collision-free, O(1) hash of (cell, block id) into the pool).
//   * The values of segment b are stored block-id-major and velocity-chunk-major: the
//     64 values of a block are 4 chunks of 16 (one vz plane of the 4x4x4 block each,
//     vx fastest), and chunk q of the block with rank r sits at float offset
//       (base[b]*4 + q*cnt[b] + r) * 16.
//     A row of cells that all hold block b is therefore one contiguous run of 64-byte
//     chunks per q, which keeps the 16-byte vector loads of a tile row coalesced.
//   * dense[b]: bit 0 = every cell has a slot for b (rank = cell index), bit 1 = every
//     cell holds b (kbits all set); sweeps skip the bitmaps when both are set.
//   * Values are float32, or bfloat16 / float16 codes q of f = q * scale[c] with one
//     power-of-two scale per chunk c (c = float offset / 16; see Codec).
#pragma once
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace vlgt {

constexpr int kChunk = 16;   // values per velocity chunk (one vz plane of a block)
constexpr int kHalo = 3;     // ghost depth of GT3: stencil 2 + one face neighbour

struct LayoutView {
    const uint64_t* ubits;
    const uint64_t* kbits;
    const uint32_t* woff;
    const uint32_t* cnt;
    const int64_t* base;
    const uint8_t* dense;
    void* pool;       // values in the grid's storage type (Codec<k>::T)
    float* scale;     // [capacity * 4] power-of-two scale of the codes of each chunk
                      // (16-bit storage; indexed like the chunks of the pool)
};

// Storage codecs.  FP32 storage keeps f.  The 16-bit forms keep q = f / s rounded to
// nearest even in bfloat16 or float16, with s the power of two of the chunk (16 values,
// one vz plane of a block) that q belongs to: dividing and multiplying by s is exact in
// FP32, so the rounding to 16 bits is the only error, and the arithmetic of a sweep stays
// FP32.  Whoever writes a chunk sets s from the largest |f| of the chunk (chunk_scale),
// so every code lies in [-1, 1] and float16 codes of a chunk of small values stay in its
// normal range however large the values elsewhere are.
template <int kCodec>
struct Codec;
template <>
struct Codec<0> {
    using T = float;
    static __device__ __forceinline__ float dec(T q, float) { return q; }
    static __device__ __forceinline__ T enc(float f, float) { return f; }
};
template <>
struct Codec<1> {
    using T = __nv_bfloat16;
    static __device__ __forceinline__ float dec(T q, float s) { return __bfloat162float(q) * s; }
    static __device__ __forceinline__ T enc(float f, float inv) { return __float2bfloat16_rn(f * inv); }
};
template <>
struct Codec<2> {
    using T = __half;
    static __device__ __forceinline__ float dec(T q, float s) { return __half2float(q) * s; }
    static __device__ __forceinline__ T enc(float f, float inv) { return __float2half_rn(f * inv); }
};

// The scale of a chunk whose largest magnitude is m, and its inverse: s is the smallest
// power of two >= m, clamped to [2^-126, 2^126] (2^-126 for an all-zero chunk), so both s
// and 1/s are normal floats and encoding (f * inv) and decoding (q * s) are exact
// scalings.  From the bit fields: adding 2^23 - 1 to the bits of a normal m carries into
// the exponent exactly when its fraction is non-zero, and clearing the fraction then
// leaves the next power of two up; s = 2^(e-127) has the inverse 2^(127-e), whose bits
// are 0x7f000000 minus those of s.
struct ChunkScale {
    float s, inv;
};
__device__ __forceinline__ ChunkScale chunk_scale(float m)
{
    const float mc = fminf(fmaxf(m, 0x1p-126f), 0x1p126f);
    const unsigned sb = (__float_as_uint(mc) + 0x007fffffu) & 0x7f800000u;
    return ChunkScale{__uint_as_float(sb), __uint_as_float(0x7f000000u - sb)};
}
// Largest value over aligned groups of `width` lanes (a power of two <= 32); every lane
// of the warp must take part.
template <int width>
__device__ __forceinline__ float group_max(float m)
{
#pragma unroll
    for (int o = width / 2; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    return m;
}

struct GridGeom {
    const int* abort;  // sticky device flag of a captured step sequence (nullptr: none);
                       // once set, every later step kernel returns at entry
    int n[3];      // nx, ny, nz
    int W;         // words per row
    int64_t R;     // rows = ny*nz
    int64_t RW;    // words per segment
    int64_t N;     // cells
    int nb;        // block ids
    int nbx, nby;  // block grid along vx, vy
};

// Per-velocity-cell constants of one sweep.  With c the Courant number v_d dt/dx_d and
// g = |c|, the mass leaving a cell through its downwind face is
//     out = g a + A minmod(d1, 2 d0) + B minmod(d0, 2 d1)
// where d0 = a - aL and d1 = aR - a are the (face-clamped) distances of the cell's
// edge values from its average.  This is the Colella-Woodward flux integral of the
// limited parabola rewritten in the edge distances (A, B follow from expanding the
// integral; for c < 0 the roles of the two faces swap).  up = 1 when content moves
// towards higher indices (inflow comes from the lower neighbour).
struct SweepConst {
    float g, A, B;
    int up;
};

__host__ __device__ inline SweepConst sweep_const(double c)
{
    SweepConst k;
    if (c >= 0.0) {
        k.g = (float)c;
        k.A = (float)(c * (1.0 - c) * (1.0 - c));
        k.B = (float)(c * c * (1.0 - c));
        k.up = 1;
    } else {
        double g = -c;
        k.g = (float)g;
        k.A = (float)(-g * g * (1.0 - g));
        k.B = (float)(-g * (1.0 - g) * (1.0 - g));
        k.up = 0;
    }
    return k;
}

// median of (x, y, 0).  It is the minmod of x and y (0 when their signs differ, else
// the one of smaller magnitude), and it is also x clamped into [min(0,y), max(0,y)].
__device__ __forceinline__ float med0(float x, float y)
{
    return fmaxf(fminf(x, y), fminf(fmaxf(x, y), 0.0f));
}

// Sign-generic PPM remap of one line, one cell average pushed per call.  After the
// value of cell p is pushed, the new average of cell p-3 is returned (the 7-cell
// dependence window p-6..p).  Face values, limiter and flux follow the oracle's
// reading of the paper (Colella-Woodward 1984 with a face value clamped between its
// two cells), evaluated in FP32 in difference form:
//   delta_j = a_{j+1} - a_j
//   e_j     = face_{j+1/2} - a_j = delta_j/2 + (delta_{j-1} - delta_{j+1})/12
//   d1_j    = e_j clamped into [min(0,delta_j), max(0,delta_j)]   (= aR_j - a_j)
//   d0_{j+1}= delta_j - d1_j                                       (= a_{j+1} - aL_{j+1})
// The CW84 limiter in these variables is d0' = minmod(d0, 2 d1), d1' = minmod(d1, 2 d0).
template <bool kLimiter>
struct Slide {
    float a1, a2, a3;  // a_{p-1}, a_{p-2}, a_{p-3}
    float l1, l2;      // delta_{p-2}, delta_{p-3}
    float d0;          // d0_{p-2}
    float o3, o4;      // out_{p-3}, out_{p-4}

    __device__ __forceinline__ void reset()
    {
        a1 = a2 = a3 = l1 = l2 = d0 = o3 = o4 = 0.0f;
    }

    __device__ __forceinline__ float push(float a, const SweepConst& k)
    {
        float dn = a - a1;                                  // delta_{p-1}
        float e = fmaf(l2 - dn, 1.0f / 12.0f, 0.5f * l1);   // e_{p-2}
        float out;
        float d1;
        if (kLimiter) {
            d1 = med0(e, l1);                               // d1_{p-2}
            float m1 = med0(d1, d0 + d0);
            float m0 = med0(d0, d1 + d1);
            out = fmaf(k.B, m0, fmaf(k.A, m1, k.g * a2));   // out_{p-2}
        } else {
            d1 = e;
            out = fmaf(k.B, d0, fmaf(k.A, d1, k.g * a2));
        }
        float res = a3 - o3 + (k.up ? o4 : out);            // new average of cell p-3
        d0 = l1 - d1;                                       // d0_{p-1}
        a3 = a2;
        a2 = a1;
        a1 = a;
        l2 = l1;
        l1 = dn;
        o4 = o3;
        o3 = out;
        return res;
    }
};

// min(|a|, |b|) carrying the sign sign(a) XOR sign(b): positive when a and b agree in
// sign, so max(result, 0) is the magnitude of minmod(a, b).
__device__ __forceinline__ float min_xorsign_abs(float a, float b)
{
    float d;
    asm("min.xorsign.abs.f32 %0, %1, %2;" : "=f"(d) : "f"(a), "f"(b));
    return d;
}

// Per-velocity-cell constants of a sweep walked in the upwind-to-downwind direction:
// in that frame c >= 0 always (a cell with c < 0 is the mirror image of one with
// c > 0), g = |c|, A = g (1-g)^2, B = g^2 (1-g).
struct WalkConst {
    float g, A, B;
    int up;  // 1: walk towards higher indices (c >= 0); 0: walk towards lower ones
};

__host__ __device__ inline WalkConst walk_const(double c)
{
    WalkConst k;
    double g = c >= 0.0 ? c : -c;
    k.g = (float)g;
    k.A = (float)(g * (1.0 - g) * (1.0 - g));
    k.B = (float)(g * g * (1.0 - g));
    k.up = c >= 0.0 ? 1 : 0;
    return k;
}

// PPM remap of one line walked from upwind to downwind, one cell average pushed per
// call; after the value of cell p (walking order) is pushed, the new average of cell
// p-2 is returned (inflow from the upwind neighbour p-3, outflow towards p-1).  Same
// reading of the paper as Slide, evaluated with the edge distances kept signed:
//   d1 = e clamped into [0, delta]  as  copysign(max(minxs(e, delta), 0), delta)
//   out = g a + sign(d1) max(A u + B w, 0),  u = minxs(d1, 2 d0), w = minxs(d0, 2 d1)
// where minxs = min_xorsign_abs.  When d0 and d1 differ in sign (a local extremum) u
// and w are <= 0 and the cell sends g a, as CW84's flattening prescribes; otherwise
// |u| = |minmod(d1, 2 d0)| and |w| = |minmod(d0, 2 d1)|.
template <bool kLimiter>
struct Walk {
    float a1, a2;  // a_{p-1}, a_{p-2}
    float l1, l2;  // delta_{p-2}, delta_{p-3}
    float d0;      // d0_{p-2}
    float o3;      // out_{p-3}

    __device__ __forceinline__ void reset()
    {
        a1 = a2 = l1 = l2 = d0 = o3 = 0.0f;
    }

    __device__ __forceinline__ float push(float a, const WalkConst& k)
    {
        float dn = a - a1;                                          // delta_{p-1}
        float e = fmaf(l2 - dn, 1.0f / 12.0f, 0.5f * l1);           // e_{p-2}
        float d1, out;
        if (kLimiter) {
            d1 = copysignf(fmaxf(min_xorsign_abs(e, l1), 0.0f), l1);
            float u = min_xorsign_abs(d1, d0 + d0);
            float w = min_xorsign_abs(d0, d1 + d1);
            float xm = fmaxf(fmaf(k.A, u, k.B * w), 0.0f);
            out = fmaf(k.g, a2, copysignf(xm, d1));                 // out_{p-2}
        } else {
            d1 = e;
            out = fmaf(k.B, d0, fmaf(k.A, d1, k.g * a2));
        }
        float res = (a2 - out) + o3;                                // new a_{p-2}
        d0 = l1 - d1;                                               // d0_{p-1}
        a2 = a1;
        a1 = a;
        l2 = l1;
        l1 = dn;
        o3 = out;
        return res;
    }
};

// Packed FP32 pairs (sm_100 family f32x2 instructions, through the compiler's float2
// builtins so that it keeps the pairs in register pairs): each lane is rounded exactly as
// the scalar add.rn / mul.rn / fma.rn, so two walks packed into one float2 give the bits
// of two scalar walks with half the floating-point instructions.  a - b is a + (-b),
// which rounds as the scalar subtraction does.
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }

__device__ __forceinline__ float2 sub2(float2 a, float2 b) { return __fadd2_rn(a, make_float2(-b.x, -b.y)); }

__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }

__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }

struct WalkConst2 {
    float2 g, A, B;
};

__device__ __forceinline__ WalkConst2 pack_const(const WalkConst& p, const WalkConst& q)
{
    return {make_float2(p.g, q.g), make_float2(p.A, q.A), make_float2(p.B, q.B)};
}

// Two Walks in lock step, lanes .x and .y; both must walk the same way.  Every
// operation is the one Walk::push performs, in the same order, per lane.
template <bool kLimiter>
struct Walk2 {
    float2 a1, a2, l1, l2, d0, o3;

    __device__ __forceinline__ void reset()
    {
        a1 = a2 = l1 = l2 = d0 = o3 = make_float2(0.0f, 0.0f);
    }

    __device__ __forceinline__ float2 push(float2 a, const WalkConst2& k)
    {
        const float2 half = make_float2(0.5f, 0.5f), twelfth = make_float2(1.0f / 12.0f, 1.0f / 12.0f);
        float2 dn = sub2(a, a1);
        float2 e = fma2(sub2(l2, dn), twelfth, mul2(half, l1));
        float2 d1, out;
        if (kLimiter) {
            d1.x = copysignf(fmaxf(min_xorsign_abs(e.x, l1.x), 0.0f), l1.x);
            d1.y = copysignf(fmaxf(min_xorsign_abs(e.y, l1.y), 0.0f), l1.y);
            const float2 dd0 = add2(d0, d0), dd1 = add2(d1, d1);
            const float2 u = make_float2(min_xorsign_abs(d1.x, dd0.x), min_xorsign_abs(d1.y, dd0.y));
            const float2 w = make_float2(min_xorsign_abs(d0.x, dd1.x), min_xorsign_abs(d0.y, dd1.y));
            float2 xm = fma2(k.A, u, mul2(k.B, w));
            xm.x = copysignf(fmaxf(xm.x, 0.0f), d1.x);
            xm.y = copysignf(fmaxf(xm.y, 0.0f), d1.y);
            out = fma2(k.g, a2, xm);
        } else {
            d1 = e;
            out = fma2(k.B, d0, fma2(k.A, d1, mul2(k.g, a2)));
        }
        float2 res = add2(sub2(a2, out), o3);
        d0 = sub2(l1, d1);
        a2 = a1;
        a1 = a;
        l2 = l1;
        l1 = dn;
        o3 = out;
        return res;
    }
};

// Slot (rank) of cell (x, row) of block id b in a layout, or -1 when the cell has no
// slot.  With check_keep the cell must also hold the block (kbits).
__device__ __forceinline__ int64_t cell_rank(const LayoutView& L, const GridGeom& G, int b,
                                             int x, int64_t row, bool check_keep)
{
    uint8_t dn = L.dense[b];
    if ((dn & 1) && (!check_keep || (dn & 2))) return row * G.n[0] + x;
    int64_t wi = (int64_t)b * G.RW + row * G.W + (x >> 6);
    uint64_t u = L.ubits[wi];
    uint64_t bit = 1ull << (x & 63);
    if (!(u & bit)) return -1;
    if (check_keep && !(L.kbits[wi] & bit)) return -1;
    return (int64_t)L.woff[wi] + __popcll(u & (bit - 1));
}

__device__ __forceinline__ int wrapi(int i, int n)
{
    int r = i % n;
    return r < 0 ? r + n : r;
}

// Device-side counters of one step (FP64 sums, block counts, error flags).
struct StepCounters {
    double mass;           // sum of all written averages (union layout)
    double dropped_mass;   // sum over removed blocks
    unsigned long long kept;
    unsigned long long dropped;
    unsigned long long work_next;  // persistent-kernel work counter (fused form)
    unsigned long long pass_next[3];  // work counters of the three passes (3-pass form)
    int error;                     // bit 2: staging wait ran out; bit 3: capacity overflow
    int done;                      // 1 once every kernel of the step has run
    long long needed;              // slots the step's union needed (capacity checks)
};

__device__ __forceinline__ bool aborted(const int* abort) { return abort && *(volatile const int*)abort; }

}  // namespace vlgt
