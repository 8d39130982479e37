// costmodel.cu -- the learned cost model of libvlgt: per-tile features of the sparse
// phase space, a small MLP (8 -> 64 -> 64 -> 1, ReLU) with its own forward, backward
// and Adam kernels, and the capacity estimate that pre-sizes the block pools of a
// captured step sequence.
//
// The paper balances its spatial cells by a weight that grows with the complexity of
// each cell's velocity space (Section 2, load balancing) and notes that the coalesced
// ghost cells change that cost (Section 5).  Here the question is the same one asked
// ahead of time on one GPU: how many blocks will a region of space hold over the next
// steps.  The model predicts, per tile of edge^3 cells, log(1 + max over a horizon of
// the tile's blocks after the 27-cell union); summed over tiles this sizes the pools.
// It never touches f: it changes only how much memory a captured sequence reserves.
//
// All reductions are deterministic (fixed summation order, FP64 accumulators), so a
// training run is reproducible bit for bit.
#include <cuda_runtime.h>
#include <stdint.h>

#include <cmath>

#include "grid.h"

namespace vlgt {

namespace {

constexpr int kIn = VL_MLP_NIN, kH = VL_MLP_NHIDDEN, kP = VL_MLP_NPARAM;
// flat parameter layout: W1[kH][kIn], b1[kH], W2[kH][kH], b2[kH], w3[kH], b3
constexpr int oW1 = 0, ob1 = oW1 + kH * kIn, oW2 = ob1 + kH, ob2 = oW2 + kH * kH, ow3 = ob2 + kH,
              ob3 = ow3 + kH;
static_assert(ob3 + 1 == kP, "parameter layout");

constexpr int kThreads = 128;
inline int nblk(int64_t n, int t) { return (int)((n + t - 1) / t); }

// ---- features ----------------------------------------------------------------------
struct TileGeom {
    GridGeom G;
    int edge;
    int nt[3];  // tiles per dimension
};

// Velocity moments of every cell for the features: one warp per 64-cell bitmap word (a
// row segment), looping over the block ids with one broadcast bitmap load each; a lane
// owns cells x and x+32 of the word.  Each present block is summed in FP32 about its own
// velocity centre v_b (offsets delta within +-1.5 dv: a = sum f, e_d = sum delta_d f,
// q_d = sum delta_d^2 f), then per cell in FP64: n = sum a, nV_d = sum (v_b,d a + e_d),
// S_d = sum (v_b,d^2 a + 2 v_b,d e_d + q_d), P_dd = S_d - (nV_d)^2 / n, all times dv^3.
// The error of P is then relative to P itself (the rounding of a block's sums enters
// with weight (v_b - V)^2), not to the much larger sum of v^2 f.
struct VMeshF {
    double vmin[3], dv[3];
};

template <int kCodec>
__global__ void __launch_bounds__(256) k_cell_moments(GridGeom G, LayoutView L, VMeshF V, double* __restrict__ mom)
{
    using C = Codec<kCodec>;
    using T = typename C::T;
    const int64_t wid = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (wid >= G.RW) return;  // warp-uniform
    const int lane = threadIdx.x & 31;
    const int64_t row = wid / G.W;
    const int w = (int)(wid - row * G.W);
    double A[2] = {0, 0}, B[2][3] = {{0, 0, 0}, {0, 0, 0}}, S[2][3] = {{0, 0, 0}, {0, 0, 0}};
    const T* pool = static_cast<const T*>(L.pool);
    for (int b = 0; b < G.nb; b++) {
        const int64_t wi = (int64_t)b * G.RW + wid;
        const uint64_t k = L.kbits[wi];
        if (!k) continue;
        const uint64_t u = L.ubits[wi];
        const int64_t wo = L.woff[wi];
        const int64_t base = L.base[b];
        const int64_t cnt = L.cnt[b];
        const bool dense = (L.dense[b] & 1) != 0;
        const int bc[3] = {b % G.nbx, (b / G.nbx) % G.nby, b / (G.nbx * G.nby)};
        double vb[3];
        for (int d = 0; d < 3; d++) vb[d] = V.vmin[d] + (4 * bc[d] + 2) * V.dv[d];
        const float dvx = (float)V.dv[0], dvy = (float)V.dv[1], dvz = (float)V.dv[2];
#pragma unroll
        for (int h = 0; h < 2; h++) {
            const int bit = lane + 32 * h;
            if (!((k >> bit) & 1ull)) continue;
            const int64_t rank = dense ? row * G.n[0] + 64 * w + bit : wo + __popcll(u & ((1ull << bit) - 1ull));
            float a = 0.f, e[3] = {0.f, 0.f, 0.f}, q[3] = {0.f, 0.f, 0.f};
#pragma unroll
            for (int iz = 0; iz < 4; iz++) {
                const int64_t chunk = base * 4 + iz * cnt + rank;
                const T* src = pool + chunk * kChunk;
                const float sc = kCodec ? L.scale[chunk] : 1.0f;
                const float dz = (iz - 1.5f) * dvz;
#pragma unroll
                for (int l = 0; l < kChunk; l++) {
                    const float f = C::dec(src[l], sc);
                    const float dx = ((l & 3) - 1.5f) * dvx, dy = ((l >> 2) - 1.5f) * dvy;
                    a += f;
                    e[0] = fmaf(dx, f, e[0]);
                    e[1] = fmaf(dy, f, e[1]);
                    e[2] = fmaf(dz, f, e[2]);
                    q[0] = fmaf(dx * dx, f, q[0]);
                    q[1] = fmaf(dy * dy, f, q[1]);
                    q[2] = fmaf(dz * dz, f, q[2]);
                }
            }
            A[h] += a;
            for (int d = 0; d < 3; d++) {
                B[h][d] += vb[d] * a + e[d];
                S[h][d] += vb[d] * vb[d] * a + 2.0 * vb[d] * e[d] + q[d];
            }
        }
    }
    const double dv3 = V.dv[0] * V.dv[1] * V.dv[2];
#pragma unroll
    for (int h = 0; h < 2; h++) {
        const int x = 64 * w + lane + 32 * h;
        if (x >= G.n[0]) continue;
        double* o = mom + (row * G.n[0] + x) * 7;
        o[0] = A[h] * dv3;
        for (int d = 0; d < 3; d++) {
            o[1 + d] = B[h][d] * dv3;
            o[4 + d] = A[h] != 0.0 ? (S[h][d] - B[h][d] * B[h][d] / A[h]) * dv3 : 0.0;
        }
    }
}

// Per tile: active blocks (kbits of the state), blocks of the next step's union (ubits
// of the next layout), and FP64 sums over the tile's cells of n, V_d, v_th and the
// relative density gradient, from the per-cell moments (n, nV_d, P_dd).
__global__ void __launch_bounds__(256) k_tile_features(TileGeom T, const uint64_t* __restrict__ kbits,
                                                       const uint64_t* __restrict__ ubits,
                                                       const double* __restrict__ mom,
                                                       float* __restrict__ feat, float* __restrict__ uni)
{
    const GridGeom& G = T.G;
    const int tile = blockIdx.x;
    const int tc[3] = {tile % T.nt[0], (tile / T.nt[0]) % T.nt[1], tile / (T.nt[0] * T.nt[1])};
    int lo[3], ext[3];
    for (int d = 0; d < 3; d++) {
        lo[d] = tc[d] * T.edge;
        ext[d] = min(T.edge, G.n[d] - lo[d]);
    }
    // block counts: (block id, tile row) pairs, the tile's x range masked in each word
    const int rows = ext[1] * ext[2];
    const int64_t pairs = (int64_t)G.nb * rows;
    unsigned long long act = 0, un = 0;
    for (int64_t i = threadIdx.x; i < pairs; i += blockDim.x) {
        const int b = (int)(i / rows);
        const int r = (int)(i - (int64_t)b * rows);
        const int64_t row = (int64_t)(lo[1] + r % ext[1]) + (int64_t)G.n[1] * (lo[2] + r / ext[1]);
        const int64_t base = (int64_t)b * G.RW + row * G.W;
        for (int x = lo[0]; x < lo[0] + ext[0];) {  // words overlapping the x range
            const int w = x >> 6;
            const int xe = min(lo[0] + ext[0], (w + 1) * 64);
            const int nbit = xe - x;
            const uint64_t m = (nbit == 64 ? ~0ull : ((1ull << nbit) - 1ull)) << (x & 63);
            act += __popcll(kbits[base + w] & m);
            un += __popcll(ubits[base + w] & m);
            x = xe;
        }
    }
    // per-cell moment features
    double s[6] = {0, 0, 0, 0, 0, 0};  // n, Vx, Vy, Vz, v_th, and (max) |grad n| / n
    const int ncell = ext[0] * ext[1] * ext[2];
    for (int c = threadIdx.x; c < ncell; c += blockDim.x) {
        const int x = lo[0] + c % ext[0], y = lo[1] + (c / ext[0]) % ext[1], z = lo[2] + c / (ext[0] * ext[1]);
        const int64_t cell = x + (int64_t)G.n[0] * (y + (int64_t)G.n[1] * z);
        const double* m = mom + cell * 7;
        const double n = m[0];
        s[0] += n;
        if (n > 0.0) {
            for (int d = 0; d < 3; d++) s[1 + d] += m[1 + d] / n;
            s[4] += sqrt((m[4] + m[5] + m[6]) / (3.0 * n));
            const int xc[3] = {x, y, z};
            double g2 = 0.0;
            for (int d = 0; d < 3; d++) {
                int up[3] = {xc[0], xc[1], xc[2]}, dn[3] = {xc[0], xc[1], xc[2]};
                up[d] = wrapi(xc[d] + 1, G.n[d]);
                dn[d] = wrapi(xc[d] - 1, G.n[d]);
                const double nu = mom[(up[0] + (int64_t)G.n[0] * (up[1] + (int64_t)G.n[1] * up[2])) * 7];
                const double nd = mom[(dn[0] + (int64_t)G.n[0] * (dn[1] + (int64_t)G.n[1] * dn[2])) * 7];
                const double gd = 0.5 * (nu - nd);
                g2 += gd * gd;
            }
            s[5] = fmax(s[5], sqrt(g2) / n);
        }
    }
    // deterministic CTA reduction: warp trees, then warps in order
    __shared__ double sh[8][6];
    __shared__ unsigned long long shc[8][2];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int o = 16; o > 0; o >>= 1) {
        for (int k = 0; k < 5; k++) s[k] += __shfl_down_sync(0xffffffffu, s[k], o);
        s[5] = fmax(s[5], __shfl_down_sync(0xffffffffu, s[5], o));
        act += __shfl_down_sync(0xffffffffu, act, o);
        un += __shfl_down_sync(0xffffffffu, un, o);
    }
    if (lane == 0) {
        for (int k = 0; k < 6; k++) sh[warp][k] = s[k];
        shc[warp][0] = act;
        shc[warp][1] = un;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double t[6] = {0, 0, 0, 0, 0, 0};
        unsigned long long A = 0, U = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); w++) {
            for (int k = 0; k < 5; k++) t[k] += sh[w][k];
            t[5] = fmax(t[5], sh[w][5]);
            A += shc[w][0];
            U += shc[w][1];
        }
        float* f = feat + (int64_t)tile * kIn;
        f[0] = (float)log1p((double)A);
        f[1] = (float)log1p((double)U);
        f[2] = (float)log1p(t[0] / ncell);
        for (int d = 0; d < 3; d++) f[3 + d] = (float)(t[1 + d] / ncell);
        f[6] = (float)(t[4] / ncell);
        f[7] = (float)t[5];
        uni[tile] = (float)U;
    }
}

// targets[t][i] = log(1 + max_{j < horizon} uni[t + j][i])
__global__ void k_cost_targets(const float* __restrict__ trace, int nsnap, int64_t ntiles, int horizon,
                               float* __restrict__ targets)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int nt = nsnap - horizon + 1;
    if (i >= (int64_t)nt * ntiles) return;
    const int t = (int)(i / ntiles);
    const int64_t k = i - (int64_t)t * ntiles;
    float m = 0.0f;
    for (int j = 0; j < horizon; j++) m = fmaxf(m, trace[(int64_t)(t + j) * ntiles + k]);
    targets[i] = (float)log1p((double)m);
}

// ---- MLP -----------------------------------------------------------------------------
__device__ __forceinline__ void load_params(const float* __restrict__ params, float* sp)
{
    for (int i = threadIdx.x; i < kP; i += blockDim.x) sp[i] = params[i];
    __syncthreads();
}

// One thread per sample: y = b3 + w3 . relu(W2 relu(W1 x + b1) + b2); the hidden
// activations are kept when h1/h2 are given (training).
__global__ void __launch_bounds__(kThreads) k_mlp_forward(const float* __restrict__ params,
                                                          const float* __restrict__ x, int64_t n,
                                                          float* __restrict__ y, float* __restrict__ h1o,
                                                          float* __restrict__ h2o)
{
    __shared__ float sp[kP];
    load_params(params, sp);
    const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n) return;
    float xi[kIn];
#pragma unroll
    for (int i = 0; i < kIn; i++) xi[i] = x[s * kIn + i];
    float h1[kH];
#pragma unroll
    for (int k = 0; k < kH; k++) {
        float a = sp[ob1 + k];
#pragma unroll
        for (int i = 0; i < kIn; i++) a = fmaf(sp[oW1 + k * kIn + i], xi[i], a);
        h1[k] = fmaxf(a, 0.0f);
        if (h1o) h1o[s * kH + k] = h1[k];
    }
    float out = sp[ob3];
    for (int j = 0; j < kH; j++) {
        float a = sp[ob2 + j];
#pragma unroll
        for (int k = 0; k < kH; k++) a = fmaf(sp[oW2 + j * kH + k], h1[k], a);
        const float h = fmaxf(a, 0.0f);
        if (h2o) h2o[s * kH + j] = h;
        out = fmaf(sp[ow3 + j], h, out);
    }
    y[s] = out;
}

// One thread per sample, loss L = (1/n) sum (y - t)^2: dL/dy, dL/d(pre-activation) of
// layer 2 (dh2) and of layer 1 (dh1); the ReLU passes the gradient where its output > 0.
__global__ void __launch_bounds__(kThreads) k_mlp_backward(const float* __restrict__ params,
                                                           const float* __restrict__ y,
                                                           const float* __restrict__ t, int64_t n,
                                                           const float* __restrict__ h1,
                                                           const float* __restrict__ h2,
                                                           float* __restrict__ dy, float* __restrict__ dh1,
                                                           float* __restrict__ dh2)
{
    __shared__ float sp[kP];
    load_params(params, sp);
    const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n) return;
    const float g = 2.0f * (y[s] - t[s]) / (float)n;
    dy[s] = g;
    float d2[kH];
#pragma unroll
    for (int j = 0; j < kH; j++) {
        d2[j] = h2[s * kH + j] > 0.0f ? g * sp[ow3 + j] : 0.0f;
        dh2[s * kH + j] = d2[j];
    }
    for (int k = 0; k < kH; k++) {
        float a = 0.0f;
        if (h1[s * kH + k] > 0.0f) {
#pragma unroll
            for (int j = 0; j < kH; j++) a = fmaf(sp[oW2 + j * kH + k], d2[j], a);
        }
        dh1[s * kH + k] = a;
    }
}

// One thread per parameter: its gradient summed over the samples in order, in FP64.
__global__ void k_mlp_param_grad(const float* __restrict__ x, const float* __restrict__ h1,
                                 const float* __restrict__ h2, const float* __restrict__ dy,
                                 const float* __restrict__ dh1, const float* __restrict__ dh2, int64_t n,
                                 float* __restrict__ grad)
{
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= kP) return;
    double acc = 0.0;
    if (p < ob1) {
        const int k = p / kIn, i = p % kIn;
        for (int64_t s = 0; s < n; s++) acc += (double)dh1[s * kH + k] * x[s * kIn + i];
    } else if (p < oW2) {
        const int k = p - ob1;
        for (int64_t s = 0; s < n; s++) acc += dh1[s * kH + k];
    } else if (p < ob2) {
        const int j = (p - oW2) / kH, k = (p - oW2) % kH;
        for (int64_t s = 0; s < n; s++) acc += (double)dh2[s * kH + j] * h1[s * kH + k];
    } else if (p < ow3) {
        const int j = p - ob2;
        for (int64_t s = 0; s < n; s++) acc += dh2[s * kH + j];
    } else if (p < ob3) {
        const int j = p - ow3;
        for (int64_t s = 0; s < n; s++) acc += (double)dy[s] * h2[s * kH + j];
    } else {
        for (int64_t s = 0; s < n; s++) acc += dy[s];
    }
    grad[p] = (float)acc;
}

// Mean squared error in FP64, one CTA, fixed order.
__global__ void k_mlp_loss(const float* __restrict__ y, const float* __restrict__ t, int64_t n, double* loss)
{
    __shared__ double sh[kThreads];
    double a = 0.0;
    for (int64_t s = threadIdx.x; s < n; s += blockDim.x) {
        const double d = (double)y[s] - t[s];
        a += d * d;
    }
    sh[threadIdx.x] = a;
    __syncthreads();
    if (threadIdx.x == 0) {
        double tot = 0.0;
        for (int i = 0; i < (int)blockDim.x; i++) tot += sh[i];
        *loss = n > 0 ? tot / (double)n : 0.0;
    }
}

// Adam (Kingma & Ba 2015) with bias correction: c1 = 1/(1 - beta1^t), c2 = 1/(1 - beta2^t).
__global__ void k_mlp_adam(float* __restrict__ params, float* __restrict__ m, float* __restrict__ v,
                           const float* __restrict__ grad, float lr, float c1, float c2)
{
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= kP) return;
    const float g = grad[p];
    const float mm = VL_MLP_BETA1 * m[p] + (1.0f - VL_MLP_BETA1) * g;
    const float vv = VL_MLP_BETA2 * v[p] + (1.0f - VL_MLP_BETA2) * g * g;
    m[p] = mm;
    v[p] = vv;
    params[p] -= lr * (mm * c1) / (sqrtf(vv * c2) + VL_MLP_EPS);
}

// capacity = ceil((1 + margin) * sum_i max(exp(y_i) - 1, 0)), FP64, one CTA, fixed order.
__global__ void k_capacity_sum(const float* __restrict__ y, int64_t n, double margin, int64_t* out)
{
    __shared__ double sh[kThreads];
    double a = 0.0;
    for (int64_t s = threadIdx.x; s < n; s += blockDim.x) a += fmax(expm1((double)y[s]), 0.0);
    sh[threadIdx.x] = a;
    __syncthreads();
    if (threadIdx.x == 0) {
        double tot = 0.0;
        for (int i = 0; i < (int)blockDim.x; i++) tot += sh[i];
        *out = (int64_t)ceil((1.0 + margin) * tot);
    }
}

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

struct TrainWs {
    float *y, *h1, *h2, *dy, *dh1, *dh2, *grad;
    double* loss;
};

size_t train_ws_layout(int64_t n, char* base, TrainWs* w)
{
    size_t o = 0;
    auto take = [&](size_t bytes) {
        char* p = base ? base + o : nullptr;
        o = align256(o + bytes);
        return p;
    };
    TrainWs t;
    t.y = (float*)take((size_t)n * 4);
    t.h1 = (float*)take((size_t)n * kH * 4);
    t.h2 = (float*)take((size_t)n * kH * 4);
    t.dy = (float*)take((size_t)n * 4);
    t.dh1 = (float*)take((size_t)n * kH * 4);
    t.dh2 = (float*)take((size_t)n * kH * 4);
    t.grad = (float*)take((size_t)kP * 4);
    t.loss = (double*)take(8);
    if (w) *w = t;
    return o;
}

vl_status launch_status()
{
    return cudaGetLastError() == cudaSuccess ? VL_OK : VL_ECUDA;
}

}  // namespace

vl_status tile_features(Grid* g, int edge, float* feat, float* uni)
{
    const GridGeom& G = g->geom;
    if (edge < 1 || edge > 64 || !feat || !uni) return fail(g, VL_EINVAL, "vl_tile_features: bad arguments");
    if (!g->has_state) return fail(g, VL_ESTATE, "vl_tile_features: no state");
    double* mom = (double*)g->alloc((size_t)G.N * 7 * 8);
    if (!mom) return fail(g, VL_ENOMEM, "vl_tile_features: scratch allocation failed");
    VMeshF V;
    for (int d = 0; d < 3; d++) {
        V.vmin[d] = g->vmesh.vmin[d];
        V.dv[d] = g->vmesh.dv[d];
    }
    const Layout& Lc = g->lay[g->cur];
    with_codec(g->codec, [&](auto c) {
        k_cell_moments<decltype(c)::value><<<nblk(G.RW * 32, 256), 256, 0, g->stream>>>(G, Lc.view(), V, mom);
    });
    note_launch();
    // the next layout's ubits become the 27-cell union of the state (the next step
    // rebuilds that layout anyway)
    launch_union(g, g->lay[g->cur], g->lay[1 - g->cur]);
    TileGeom T;
    T.G = G;
    T.edge = edge;
    int64_t ntiles = 1;
    for (int d = 0; d < 3; d++) {
        T.nt[d] = (G.n[d] + edge - 1) / edge;
        ntiles *= T.nt[d];
    }
    k_tile_features<<<(unsigned)ntiles, 256, 0, g->stream>>>(T, g->lay[g->cur].kbits, g->lay[1 - g->cur].ubits,
                                                             mom, feat, uni);
    note_launch();
    cudaError_t e = cudaStreamSynchronize(g->stream);
    g->release(mom);
    return e == cudaSuccess ? VL_OK : cuda_fail(g, e, "vl_tile_features");
}

}  // namespace vlgt

using namespace vlgt;

extern "C" int64_t vl_tile_count(const vl_space_desc* space, int edge)
{
    if (!space || edge < 1) return -1;
    int64_t t = 1;
    for (int d = 0; d < 3; d++) t *= (space->n[d] + edge - 1) / edge;
    return t;
}

extern "C" vl_status vl_cost_targets(const float* union_trace, int nsnap, int64_t ntiles, int horizon,
                                     float* targets, void* stream)
{
    if (!union_trace || !targets || ntiles < 0 || horizon < 1 || nsnap < horizon) return VL_EINVAL;
    const int64_t n = (int64_t)(nsnap - horizon + 1) * ntiles;
    if (n == 0) return VL_OK;
    k_cost_targets<<<nblk(n, 256), 256, 0, (cudaStream_t)stream>>>(union_trace, nsnap, ntiles, horizon, targets);
    note_launch();
    return launch_status();
}

extern "C" vl_status vl_mlp_forward(const float* params, const float* x, int64_t n, float* y, void* stream)
{
    if (!params || n < 0 || (n > 0 && (!x || !y))) return VL_EINVAL;
    if (n == 0) return VL_OK;
    k_mlp_forward<<<nblk(n, kThreads), kThreads, 0, (cudaStream_t)stream>>>(params, x, n, y, nullptr, nullptr);
    note_launch();
    return launch_status();
}

extern "C" size_t vl_mlp_workspace_bytes(int64_t n)
{
    return n < 0 ? 0 : train_ws_layout(n, nullptr, nullptr);
}

extern "C" vl_status vl_mlp_train_step(float* params, float* adam_m, float* adam_v, const float* x,
                                       const float* t, int64_t n, int step, float lr, void* workspace,
                                       size_t workspace_bytes, double* loss, void* stream)
{
    if (!params || !adam_m || !adam_v || !x || !t || n <= 0 || step < 1 || !(lr >= 0.0f) || !workspace)
        return VL_EINVAL;
    if (workspace_bytes < train_ws_layout(n, nullptr, nullptr) || ((uintptr_t)workspace & 255)) return VL_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    TrainWs w;
    train_ws_layout(n, static_cast<char*>(workspace), &w);
    const int nb = nblk(n, kThreads);
    k_mlp_forward<<<nb, kThreads, 0, s>>>(params, x, n, w.y, w.h1, w.h2);
    k_mlp_loss<<<1, kThreads, 0, s>>>(w.y, t, n, w.loss);
    k_mlp_backward<<<nb, kThreads, 0, s>>>(params, w.y, t, n, w.h1, w.h2, w.dy, w.dh1, w.dh2);
    k_mlp_param_grad<<<nblk(kP, kThreads), kThreads, 0, s>>>(x, w.h1, w.h2, w.dy, w.dh1, w.dh2, n, w.grad);
    const double c1 = 1.0 / (1.0 - std::pow((double)VL_MLP_BETA1, step));
    const double c2 = 1.0 / (1.0 - std::pow((double)VL_MLP_BETA2, step));
    k_mlp_adam<<<nblk(kP, kThreads), kThreads, 0, s>>>(params, adam_m, adam_v, w.grad, lr, (float)c1, (float)c2);
    for (int i = 0; i < 5; i++) note_launch();
    if (loss) cudaMemcpyAsync(loss, w.loss, 8, cudaMemcpyDeviceToDevice, s);
    return launch_status();
}

extern "C" vl_status vl_mlp_gradient(const float* params, const float* x, const float* t, int64_t n,
                                     void* workspace, size_t workspace_bytes, float* grad, double* loss,
                                     void* stream)
{
    if (!params || !x || !t || n <= 0 || !workspace || !grad) return VL_EINVAL;
    if (workspace_bytes < train_ws_layout(n, nullptr, nullptr) || ((uintptr_t)workspace & 255)) return VL_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    TrainWs w;
    train_ws_layout(n, static_cast<char*>(workspace), &w);
    const int nb = nblk(n, kThreads);
    k_mlp_forward<<<nb, kThreads, 0, s>>>(params, x, n, w.y, w.h1, w.h2);
    k_mlp_loss<<<1, kThreads, 0, s>>>(w.y, t, n, w.loss);
    k_mlp_backward<<<nb, kThreads, 0, s>>>(params, w.y, t, n, w.h1, w.h2, w.dy, w.dh1, w.dh2);
    k_mlp_param_grad<<<nblk(kP, kThreads), kThreads, 0, s>>>(x, w.h1, w.h2, w.dy, w.dh1, w.dh2, n, grad);
    for (int i = 0; i < 4; i++) note_launch();
    if (loss) cudaMemcpyAsync(loss, w.loss, 8, cudaMemcpyDeviceToDevice, s);
    return launch_status();
}

extern "C" vl_status vl_mlp_capacity(const float* params, const float* features, int64_t ntiles,
                                     double margin, void* workspace, size_t workspace_bytes,
                                     int64_t* capacity, void* stream)
{
    if (!params || !features || ntiles <= 0 || !workspace || !capacity || !(margin >= 0.0)) return VL_EINVAL;
    if (workspace_bytes < align256((size_t)ntiles * 4) + 8 || ((uintptr_t)workspace & 255)) return VL_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    float* y = static_cast<float*>(workspace);
    int64_t* out = reinterpret_cast<int64_t*>(static_cast<char*>(workspace) + align256((size_t)ntiles * 4));
    k_mlp_forward<<<nblk(ntiles, kThreads), kThreads, 0, s>>>(params, features, ntiles, y, nullptr, nullptr);
    k_capacity_sum<<<1, kThreads, 0, s>>>(y, ntiles, margin, out);
    note_launch();
    note_launch();
    cudaError_t e = cudaMemcpyAsync(capacity, out, 8, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    return e == cudaSuccess ? VL_OK : VL_ECUDA;
}
