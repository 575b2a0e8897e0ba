// Learned warm start for the variable-coefficient Poisson CG: a 4-layer,
// 32-channel, 3x3 (dilated) convolutional network mapping (log k, f) -> u,
// with hand-written forward, backward and Adam kernels.  Not in the paper;
// plain CG to the same tolerance still decides when every solve is done.
//
// Layers: conv(2->C) ReLU, conv(C->C) ReLU, conv(C->C) ReLU, conv(C->1);
// dilation per layer; zero padding.  Activations are stored in bf16 (or
// fp32), every product is accumulated in fp32, master weights are fp32.
// Backward through a layer: the input gradient is the same direct
// convolution with the weights flipped and transposed, masked by the ReLU of
// the forward activation; the weight gradient accumulates, per block, over a
// strided set of pixel tiles in registers before one atomic add per weight.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <type_traits>
#include <vector>

#include "common.cuh"
#include "internal.h"
#include "warmnet_tc.cuh"

using namespace perks;

namespace {

constexpr int kTile = 16;        // output pixels per block side
constexpr int kConvThreads = kTile * kTile;
constexpr int kMaxC = 32;

template <typename S> __device__ __forceinline__ float ld_f(const S *p) { return to_acc(*p); }
template <> __device__ __forceinline__ float ld_f<float>(const float *p) { return *p; }
template <typename S> __device__ __forceinline__ S st_f(float v) { return from_acc<S>(v); }
template <> __device__ __forceinline__ float st_f<float>(float v) { return v; }

// out[img][co][y][x] = bias[co] + sum_ci sum_tap W'[ci][tap][co] in[img][ci][y+dy][x+dx]
// W' is gathered from the layer weights w[cout_l][cin_l][9]:
//   TRANSPOSE = false: W'[ci][tap][co] = w[co][ci][tap]        (forward)
//   TRANSPOSE = true : W'[ci][tap][co] = w[ci][co][8 - tap]    (input gradient)
// Epilogue: RELU -> max(0, .); MASK -> multiply by (mask[img][co][p] > 0).
template <typename SI, typename SO, int CIN, int COUT, bool TRANSPOSE, bool RELU, bool MASK, typename SM>
__global__ void __launch_bounds__(kConvThreads) conv_kernel(const SI *__restrict__ in, const float *__restrict__ w,
                                                          const float *__restrict__ bias, SO *__restrict__ out,
                                                          const SM *__restrict__ mask, int H, int W, int dil,
                                                          int tiles_x, int tiles_y) {
    extern __shared__ __align__(16) float smem[];
    const int halo = dil;
    const int TW = kTile + 2 * halo;
    float *s_w = smem;                           // CIN * 9 * COUT
    float *s_in = smem + CIN * 9 * COUT;         // CIN * TW * TW
    const int tile = blockIdx.x;
    const int img = blockIdx.y;
    const int tx0 = (tile % tiles_x) * kTile, ty0 = (tile / tiles_x) * kTile;
    for (int e = threadIdx.x; e < CIN * 9 * COUT; e += blockDim.x) {
        const int co = e % COUT, tap = (e / COUT) % 9, ci = e / (9 * COUT);
        s_w[e] = TRANSPOSE ? w[(ci * COUT + co) * 9 + (8 - tap)] : w[(co * CIN + ci) * 9 + tap];
    }
    const long long plane = (long long)H * W;
    const SI *inb = in + (long long)img * CIN * plane;
    for (int e = threadIdx.x; e < CIN * TW * TW; e += blockDim.x) {
        const int xx = e % TW, yy = (e / TW) % TW, ci = e / (TW * TW);
        const int gx = tx0 + xx - halo, gy = ty0 + yy - halo;
        s_in[e] = (gx >= 0 && gx < W && gy >= 0 && gy < H) ? ld_f(inb + ci * plane + (long long)gy * W + gx) : 0.f;
    }
    __syncthreads();
    const int lx = threadIdx.x % kTile, ly = threadIdx.x / kTile;
    const int gx = tx0 + lx, gy = ty0 + ly;
    float acc[COUT];
#pragma unroll
    for (int co = 0; co < COUT; ++co) acc[co] = bias ? bias[co] : 0.f;
    for (int ci = 0; ci < CIN; ++ci) {
#pragma unroll
        for (int tap = 0; tap < 9; ++tap) {
            const int ky = tap / 3, kx = tap % 3;
            const float v = s_in[(ci * TW + ly + ky * dil) * TW + lx + kx * dil];
            const float *wr = s_w + (ci * 9 + tap) * COUT;
#pragma unroll
            for (int co = 0; co < COUT; ++co) acc[co] = fmaf(wr[co], v, acc[co]);
        }
    }
    if (gx < W && gy < H) {
        SO *ob = out + (long long)img * COUT * plane + (long long)gy * W + gx;
        const SM *mb = MASK ? mask + (long long)img * COUT * plane + (long long)gy * W + gx : nullptr;
#pragma unroll
        for (int co = 0; co < COUT; ++co) {
            float v = acc[co];
            if (RELU) v = fmaxf(v, 0.f);
            if (MASK) v = ld_f(mb + co * plane) > 0.f ? v : 0.f;
            ob[co * plane] = st_f<SO>(v);
        }
    }
}

// dW[co][ci][tap] += sum_{img,p} dy[img][co][p] * x[img][ci][p + off(tap)],
// db[co] += sum dy[img][co][p].  Thread t < CIN*9 owns (ci, tap) for all co.
template <typename SX, int CIN, int COUT>
__global__ void __launch_bounds__(kMaxC * 9) wgrad_kernel(const SX *__restrict__ x, const float *__restrict__ dy,
                                                          float *dw, float *db, int nimg, int H, int W, int dil,
                                                          int tiles_x, int tiles_y) {
    extern __shared__ __align__(16) float smem[];
    const int halo = dil;
    const int TW = kTile + 2 * halo;
    float *s_x = smem;                          // CIN * TW * TW
    float *s_dy = smem + CIN * TW * TW;         // kTile*kTile * COUT, [p][co]
    const int t = threadIdx.x;
    const bool active = t < CIN * 9;
    const int ci = active ? t / 9 : 0, tap = active ? t % 9 : 0;
    const int ky = tap / 3, kx = tap % 3;
    float acc[COUT];
    float bacc = 0.f;
#pragma unroll
    for (int co = 0; co < COUT; ++co) acc[co] = 0.f;
    const long long plane = (long long)H * W;
    const int ntile = tiles_x * tiles_y;
    for (long long job = blockIdx.x; job < (long long)ntile * nimg; job += gridDim.x) {
        const int img = (int)(job / ntile), tile = (int)(job % ntile);
        const int tx0 = (tile % tiles_x) * kTile, ty0 = (tile / tiles_x) * kTile;
        __syncthreads();
        const SX *xb = x + (long long)img * CIN * plane;
        for (int e = t; e < CIN * TW * TW; e += blockDim.x) {
            const int xx = e % TW, yy = (e / TW) % TW, c = e / (TW * TW);
            const int gx = tx0 + xx - halo, gy = ty0 + yy - halo;
            s_x[e] = (gx >= 0 && gx < W && gy >= 0 && gy < H) ? ld_f(xb + c * plane + (long long)gy * W + gx) : 0.f;
        }
        const float *dyb = dy + (long long)img * COUT * plane;
        for (int e = t; e < kTile * kTile * COUT; e += blockDim.x) {
            const int co = e % COUT, p = e / COUT;
            const int gx = tx0 + p % kTile, gy = ty0 + p / kTile;
            s_dy[e] = (gx < W && gy < H) ? dyb[co * plane + (long long)gy * W + gx] : 0.f;
        }
        __syncthreads();
        if (active) {
            for (int p = 0; p < kTile * kTile; ++p) {
                const int py = p / kTile, px = p % kTile;
                const float v = s_x[(ci * TW + py + ky * dil) * TW + px + kx * dil];
                const float *d = s_dy + p * COUT;
#pragma unroll
                for (int co = 0; co < COUT; ++co) acc[co] = fmaf(d[co], v, acc[co]);
            }
        }
        if (t < COUT)
            for (int p = 0; p < kTile * kTile; ++p) bacc += s_dy[p * COUT + t];
    }
    if (active) {
#pragma unroll
        for (int co = 0; co < COUT; ++co) atomicAdd(dw + (co * CIN + ci) * 9 + tap, acc[co]);
    }
    if (t < COUT) atomicAdd(db + t, bacc);
}

// Network input: channel 0 = log k, channel 1 = f, each averaged over the
// F x F fine cells of a coarse cell (F = 1: the cells themselves).
template <typename S>
__global__ void features_kernel(const double *__restrict__ k, const double *__restrict__ f, S *x0, int ny, int nx,
                                int F, int nimg) {
    const int H = ny / F, W = nx / F;
    const long long plane = (long long)H * W;
    const double inv = 1.0 / ((double)F * F);
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < plane * nimg;
         i += (long long)gridDim.x * blockDim.x) {
        const long long img = i / plane, p = i % plane;
        const int Y = (int)(p / W), X = (int)(p % W);
        double lk = 0.0, ff = 0.0;
        for (int dy = 0; dy < F; ++dy)
            for (int dx = 0; dx < F; ++dx) {
                const long long c = (img * ny + (long long)Y * F + dy) * nx + (long long)X * F + dx;
                lk += log(k[c]);
                ff += f[c];
            }
        x0[(img * 2 + 0) * plane + p] = st_f<S>((float)(lk * inv));
        x0[(img * 2 + 1) * plane + p] = st_f<S>((float)(ff * inv));
    }
}

// Mean of u over each F x F block (training target at the network's grid).
__global__ void pool_kernel(const double *__restrict__ u, double *ut, int ny, int nx, int F, int nimg) {
    const int H = ny / F, W = nx / F;
    const long long plane = (long long)H * W;
    const double inv = 1.0 / ((double)F * F);
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < plane * nimg;
         i += (long long)gridDim.x * blockDim.x) {
        const long long img = i / plane, p = i % plane;
        const int Y = (int)(p / W), X = (int)(p % W);
        double acc = 0.0;
        for (int dy = 0; dy < F; ++dy)
            for (int dx = 0; dx < F; ++dx) acc += u[(img * ny + (long long)Y * F + dy) * nx + (long long)X * F + dx];
        ut[i] = acc * inv;
    }
}

// u = scale * bilinear interpolation of the coarse output at the fine cell
// centres (coarse cell centres at (Y + 1/2) F - 1/2, clamped at the edges).
__global__ void upsample_kernel(const float *__restrict__ out, float scale, int ny, int nx, int F, int nimg,
                                double *u) {
    const int H = ny / F, W = nx / F;
    const long long total = (long long)nimg * ny * nx;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const long long img = i / ((long long)ny * nx), p = i % ((long long)ny * nx);
        const int y = (int)(p / nx), x = (int)(p % nx);
        double yc = (y + 0.5) / F - 0.5, xc = (x + 0.5) / F - 0.5;
        yc = fmin(fmax(yc, 0.0), (double)(H - 1));
        xc = fmin(fmax(xc, 0.0), (double)(W - 1));
        const int y0 = (int)yc, x0 = (int)xc;
        const int y1 = min(y0 + 1, H - 1), x1 = min(x0 + 1, W - 1);
        const double wy = yc - y0, wx = xc - x0;
        const float *o = out + img * (long long)H * W;
        const double v = (1.0 - wy) * ((1.0 - wx) * o[(long long)y0 * W + x0] + wx * o[(long long)y0 * W + x1]) +
                         wy * ((1.0 - wx) * o[(long long)y1 * W + x0] + wx * o[(long long)y1 * W + x1]);
        u[i] = v * scale;
    }
}

// dout = 2 (out - u/scale) / N; loss += (out - u/scale)^2 / N
__global__ void mse_kernel(const float *__restrict__ out, const double *__restrict__ u, float inv_scale,
                           long long n, float *dout, float *loss) {
    __shared__ float red[32];
    float s = 0.f;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const float d = out[i] - (float)u[i] * inv_scale;
        dout[i] = 2.f * d / (float)n;
        s = fmaf(d, d, s);
    }
    s = warp_sum(s);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x < 32) {
        float v = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.f;
        v = warp_sum(v);
        if (threadIdx.x == 0) atomicAdd(loss, v / (float)n);
    }
}

// sum of u^2 over n values into *acc (fp64)
__global__ void sumsq_kernel(const double *__restrict__ u, long long n, double *acc) {
    __shared__ double red[32];
    double s = 0.0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        s = fma(u[i], u[i], s);
    s = warp_sum(s);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x < 32) {
        double v = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0;
        v = warp_sum(v);
        if (threadIdx.x == 0) atomicAdd(acc, v);
    }
}

__global__ void to_u_kernel(const float *__restrict__ out, float scale, long long n, double *u) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        u[i] = (double)out[i] * scale;
}

__global__ void adam_kernel(float *p, const float *g, float *m, float *v, int n, float lr, float b1, float b2,
                            float eps, float c1, float c2) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

size_t conv_smem(int cin, int cout, int dil) {
    const int TW = kTile + 2 * dil;
    return sizeof(float) * ((size_t)cin * 9 * cout + (size_t)cin * TW * TW);
}
size_t wgrad_smem(int cin, int cout, int dil) {
    const int TW = kTile + 2 * dil;
    return sizeof(float) * ((size_t)cin * TW * TW + (size_t)kTile * kTile * cout);
}

template <typename K> perks_status set_smem(perks_context *ctx, K kernel, size_t bytes) {
    PERKS_CUDA(ctx, cudaFuncSetAttribute((const void *)kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
    return PERKS_OK;
}

}  // namespace

struct perks_warmnet {
    perks_context *ctx = nullptr;
    int device = 0;  // for destroy, which may come after the context is gone
    int C = kMaxC;
    int dil[4] = {1, 2, 4, 8};
    int storage = PERKS_BF16;
    float out_scale = 1.f;
    int pool = 1;                // the network runs on the grid coarsened by this factor
    bool tensor_cores = true;    // bf16 storage: inner layers on tcgen05 (else CUDA cores)
    DevError *err = nullptr;
    double *ut = nullptr;        // pooled training target
    long long cap_ut = 0;
    int nparams = 0;
    int off_w[4], off_b[4];
    float *params = nullptr, *grads = nullptr, *m = nullptr, *v = nullptr;
    long long adam_t = 0;
    float *loss = nullptr;
    // activations, sized for the largest batch seen
    long long cap_pixels = 0;   // nimg * H * W
    void *x0 = nullptr, *x1 = nullptr, *x2 = nullptr, *x3 = nullptr;
    float *outb = nullptr, *g0 = nullptr, *g1 = nullptr;
};

namespace {

void free_net_bufs(perks_warmnet *n) {
    void *p[] = {n->x0, n->x1, n->x2, n->x3, n->outb, n->g0, n->g1};
    for (void *q : p) if (q) cudaFree(q);
    n->x0 = n->x1 = n->x2 = n->x3 = nullptr;
    n->outb = n->g0 = n->g1 = nullptr;
    n->cap_pixels = 0;
}

perks_status ensure_bufs(perks_warmnet *n, long long pixels) {
    if (pixels <= n->cap_pixels) return PERKS_OK;
    free_net_bufs(n);
    const size_t es = n->storage == PERKS_BF16 ? 2 : 4;
    perks_context *ctx = n->ctx;
    PERKS_CUDA(ctx, cudaMalloc(&n->x0, pixels * 2 * es));
    PERKS_CUDA(ctx, cudaMalloc(&n->x1, pixels * n->C * es));
    PERKS_CUDA(ctx, cudaMalloc(&n->x2, pixels * n->C * es));
    PERKS_CUDA(ctx, cudaMalloc(&n->x3, pixels * n->C * es));
    PERKS_CUDA(ctx, cudaMalloc(&n->outb, pixels * sizeof(float)));
    PERKS_CUDA(ctx, cudaMalloc(&n->g0, pixels * n->C * sizeof(float)));
    PERKS_CUDA(ctx, cudaMalloc(&n->g1, pixels * n->C * sizeof(float)));
    n->cap_pixels = pixels;
    return PERKS_OK;
}

// Forward pass on nimg fine images of ny x nx cells: features pooled to the
// network grid H x W = (ny / pool) x (nx / pool), output left in outb.
template <typename S>
perks_status forward(perks_warmnet *n, int nimg, int ny, int nx, const double *k, const double *f, cudaStream_t s) {
    perks_context *ctx = n->ctx;
    const int H = ny / n->pool, W = nx / n->pool;
    const int tx = (W + kTile - 1) / kTile, ty = (H + kTile - 1) / kTile;
    const dim3 grid(tx * ty, nimg);
    S *x0 = (S *)n->x0, *x1 = (S *)n->x1, *x2 = (S *)n->x2, *x3 = (S *)n->x3;
    features_kernel<S><<<1024, 256, 0, s>>>(k, f, x0, ny, nx, n->pool, nimg);
    const float *P = n->params;
    {
        auto kern = conv_kernel<S, S, 2, kMaxC, false, true, false, float>;
        const size_t sm = conv_smem(2, kMaxC, n->dil[0]);
        perks_status rc = set_smem(ctx, kern, sm);
        if (rc) return rc;
        kern<<<grid, kConvThreads, sm, s>>>(x0, P + n->off_w[0], P + n->off_b[0], x1, (const float *)nullptr, H, W,
                                           n->dil[0], tx, ty);
    }
    if (std::is_same<S, __nv_bfloat16>::value && n->tensor_cores) {
        // inner layers as implicit GEMMs on the tensor cores
        perks_status rc = set_smem(ctx, tc_conv32_kernel, tc_conv_smem());
        if (rc) return rc;
        const long long ntiles = (long long)nimg * (((long long)H * W + kTcPix - 1) / kTcPix);
        const int blocks = (int)std::min<long long>(ntiles, 2LL * ctx->sm_count);
        for (int l = 1; l <= 2; ++l)
            tc_conv32_kernel<<<blocks, kTcThreads, tc_conv_smem(), s>>>(
                reinterpret_cast<const __nv_bfloat16 *>(l == 1 ? x1 : x2), P + n->off_w[l], P + n->off_b[l],
                reinterpret_cast<__nv_bfloat16 *>(l == 1 ? x2 : x3), nimg, H, W, n->dil[l], n->err);
    } else {
        auto kern = conv_kernel<S, S, kMaxC, kMaxC, false, true, false, float>;
        for (int l = 1; l <= 2; ++l) {
            const size_t sm = conv_smem(kMaxC, kMaxC, n->dil[l]);
            perks_status rc = set_smem(ctx, kern, sm);
            if (rc) return rc;
            kern<<<grid, kConvThreads, sm, s>>>(l == 1 ? x1 : x2, P + n->off_w[l], P + n->off_b[l], l == 1 ? x2 : x3,
                                               (const float *)nullptr, H, W, n->dil[l], tx, ty);
        }
    }
    {
        auto kern = conv_kernel<S, float, kMaxC, 1, false, false, false, float>;
        const size_t sm = conv_smem(kMaxC, 1, n->dil[3]);
        perks_status rc = set_smem(ctx, kern, sm);
        if (rc) return rc;
        kern<<<grid, kConvThreads, sm, s>>>(x3, P + n->off_w[3], P + n->off_b[3], n->outb, (const float *)nullptr, H,
                                           W, n->dil[3], tx, ty);
    }
    PERKS_CUDA(ctx, cudaGetLastError());
    return PERKS_OK;
}

template <typename S>
perks_status backward(perks_warmnet *n, int nimg, int H, int W, cudaStream_t s) {
    perks_context *ctx = n->ctx;
    const int tx = (W + kTile - 1) / kTile, ty = (H + kTile - 1) / kTile;
    const dim3 grid(tx * ty, nimg);
    const int wgrid = 4 * ctx->sm_count;
    S *x0 = (S *)n->x0, *x1 = (S *)n->x1, *x2 = (S *)n->x2, *x3 = (S *)n->x3;
    const float *P = n->params;
    float *G = n->grads;
    PERKS_CUDA(ctx, cudaMemsetAsync(G, 0, sizeof(float) * n->nparams, s));
    // layer 4 (C -> 1): dy = outb-gradient in g1[0..pixels)
    float *dy4 = n->g1;
    {
        auto kw = wgrad_kernel<S, kMaxC, 1>;
        const size_t sm = wgrad_smem(kMaxC, 1, n->dil[3]);
        perks_status rc = set_smem(ctx, kw, sm);
        if (rc) return rc;
        kw<<<wgrid, kMaxC * 9, sm, s>>>(x3, dy4, G + n->off_w[3], G + n->off_b[3], nimg, H, W, n->dil[3], tx, ty);
        auto kd = conv_kernel<float, float, 1, kMaxC, true, false, true, S>;
        const size_t sd = conv_smem(1, kMaxC, n->dil[3]);
        rc = set_smem(ctx, kd, sd);
        if (rc) return rc;
        kd<<<grid, kConvThreads, sd, s>>>(dy4, P + n->off_w[3], nullptr, n->g0, x3, H, W, n->dil[3], tx, ty);
    }
    // layers 3 and 2 (C -> C)
    float *dy = n->g0, *dx = n->g1;
    for (int l = 2; l >= 1; --l) {
        S *xin = l == 2 ? x2 : x1;
        auto kw = wgrad_kernel<S, kMaxC, kMaxC>;
        const size_t sm = wgrad_smem(kMaxC, kMaxC, n->dil[l]);
        perks_status rc = set_smem(ctx, kw, sm);
        if (rc) return rc;
        kw<<<wgrid, kMaxC * 9, sm, s>>>(xin, dy, G + n->off_w[l], G + n->off_b[l], nimg, H, W, n->dil[l], tx, ty);
        auto kd = conv_kernel<float, float, kMaxC, kMaxC, true, false, true, S>;
        const size_t sd = conv_smem(kMaxC, kMaxC, n->dil[l]);
        rc = set_smem(ctx, kd, sd);
        if (rc) return rc;
        kd<<<grid, kConvThreads, sd, s>>>(dy, P + n->off_w[l], nullptr, dx, xin, H, W, n->dil[l], tx, ty);
        float *t = dy; dy = dx; dx = t;
    }
    // layer 1 (2 -> C): weight gradient only
    {
        auto kw = wgrad_kernel<S, 2, kMaxC>;
        const size_t sm = wgrad_smem(2, kMaxC, n->dil[0]);
        perks_status rc = set_smem(ctx, kw, sm);
        if (rc) return rc;
        kw<<<wgrid, kMaxC * 9, sm, s>>>(x0, dy, G + n->off_w[0], G + n->off_b[0], nimg, H, W, n->dil[0], tx, ty);
    }
    PERKS_CUDA(ctx, cudaGetLastError());
    return PERKS_OK;
}

// SplitMix64 -> normal (Box-Muller) for the He initialisation.
struct Rng {
    uint64_t s;
    uint64_t next() {
        uint64_t z = (s += 0x9E3779B97F4A7C15ull);
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        return z ^ (z >> 31);
    }
    double uniform() { return (double)(next() >> 11) * (1.0 / 9007199254740992.0); }
    double normal() {
        const double u1 = std::max(uniform(), 1e-300), u2 = uniform();
        return std::sqrt(-2.0 * std::log(u1)) * std::cos(6.283185307179586 * u2);
    }
};

perks_status loss_and_grad(perks_warmnet *n, int nimg, int ny, int nx, const double *k, const double *f,
                           const double *u, cudaStream_t s) {
    perks_context *ctx = n->ctx;
    const int H = ny / n->pool, W = nx / n->pool;
    const long long pixels = (long long)nimg * H * W;
    perks_status rc = ensure_bufs(n, pixels);
    if (rc) return rc;
    const double *target = u;
    if (n->pool > 1) {
        if (pixels > n->cap_ut) {
            if (n->ut) cudaFree(n->ut);
            n->ut = nullptr;
            n->cap_ut = 0;
            PERKS_CUDA(ctx, cudaMalloc(&n->ut, sizeof(double) * pixels));
            n->cap_ut = pixels;
        }
        pool_kernel<<<1024, 256, 0, s>>>(u, n->ut, ny, nx, n->pool, nimg);
        target = n->ut;
    }
    rc = n->storage == PERKS_BF16 ? forward<__nv_bfloat16>(n, nimg, ny, nx, k, f, s)
                                  : forward<float>(n, nimg, ny, nx, k, f, s);
    if (rc) return rc;
    PERKS_CUDA(ctx, cudaMemsetAsync(n->loss, 0, sizeof(float), s));
    mse_kernel<<<1024, 256, 0, s>>>(n->outb, target, 1.f / n->out_scale, pixels, n->g1, n->loss);
    PERKS_CUDA(ctx, cudaGetLastError());
    return n->storage == PERKS_BF16 ? backward<__nv_bfloat16>(n, nimg, H, W, s) : backward<float>(n, nimg, H, W, s);
}

}  // namespace

// ======================================================================= ABI

extern "C" perks_status perks_warmnet_create(perks_context *ctx, const int32_t *dilations, int32_t storage,
                                             uint64_t seed, perks_warmnet **out) {
    if (!ctx) return PERKS_ERR_INVALID_ARG;
    if (!out || (storage != PERKS_BF16 && storage != PERKS_F32))
        return fail(ctx, PERKS_ERR_INVALID_ARG, "warmnet_create: storage must be BF16 or F32");
    *out = nullptr;
    perks_status rc = use_device(ctx);
    if (rc) return rc;
    auto *n = new perks_warmnet();
    n->ctx = ctx;
    n->device = ctx->device;
    n->storage = storage;
    if (dilations)
        for (int l = 0; l < 4; ++l) {
            if (dilations[l] < 1 || dilations[l] > 16) { delete n; return fail(ctx, PERKS_ERR_INVALID_ARG, "warmnet_create: dilation in 1..16"); }
            n->dil[l] = dilations[l];
        }
    const int cins[4] = {2, n->C, n->C, n->C}, couts[4] = {n->C, n->C, n->C, 1};
    int o = 0;
    std::vector<float> h;
    Rng rng{seed};
    for (int l = 0; l < 4; ++l) {
        n->off_w[l] = o;
        const int nw = couts[l] * cins[l] * 9;
        const double sd = std::sqrt(2.0 / (cins[l] * 9.0));
        for (int i = 0; i < nw; ++i) h.push_back((float)(sd * rng.normal()));
        o += nw;
        n->off_b[l] = o;
        for (int i = 0; i < couts[l]; ++i) h.push_back(0.f);
        o += couts[l];
    }
    n->nparams = o;
    cudaError_t e = cudaMalloc(&n->params, sizeof(float) * o);
    if (e == cudaSuccess) e = cudaMalloc(&n->grads, sizeof(float) * o);
    if (e == cudaSuccess) e = cudaMalloc(&n->m, sizeof(float) * o);
    if (e == cudaSuccess) e = cudaMalloc(&n->v, sizeof(float) * o);
    if (e == cudaSuccess) e = cudaMalloc(&n->loss, sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&n->err, sizeof(DevError));
    if (e == cudaSuccess) e = cudaMemset(n->err, 0, sizeof(DevError));
    if (e == cudaSuccess) e = cudaMemcpy(n->params, h.data(), sizeof(float) * o, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(n->m, 0, sizeof(float) * o);
    if (e == cudaSuccess) e = cudaMemset(n->v, 0, sizeof(float) * o);
    if (e != cudaSuccess) { perks_warmnet_destroy(n); return cuda_fail(ctx, e, "warmnet_create"); }
    *out = n;
    return PERKS_OK;
}

extern "C" perks_status perks_warmnet_destroy(perks_warmnet *n) {
    if (!n) return PERKS_OK;
    cudaSetDevice(n->device);
    free_net_bufs(n);
    void *p[] = {n->params, n->grads, n->m, n->v, n->loss, n->ut, n->err};
    for (void *q : p) if (q) cudaFree(q);
    delete n;
    return PERKS_OK;
}

extern "C" int32_t perks_warmnet_num_params(const perks_warmnet *n) { return n ? n->nparams : 0; }

extern "C" perks_status perks_warmnet_get_params(perks_warmnet *n, float *host) {
    if (!n || !host) return PERKS_ERR_INVALID_ARG;
    PERKS_CUDA(n->ctx, cudaMemcpy(host, n->params, sizeof(float) * n->nparams, cudaMemcpyDeviceToHost));
    return PERKS_OK;
}

extern "C" perks_status perks_warmnet_set_params(perks_warmnet *n, const float *host) {
    if (!n || !host) return PERKS_ERR_INVALID_ARG;
    PERKS_CUDA(n->ctx, cudaMemcpy(n->params, host, sizeof(float) * n->nparams, cudaMemcpyHostToDevice));
    return PERKS_OK;
}

extern "C" perks_status perks_warmnet_set_scale(perks_warmnet *n, float out_scale) {
    if (!n || !(out_scale > 0.f)) return PERKS_ERR_INVALID_ARG;
    n->out_scale = out_scale;
    return PERKS_OK;
}

extern "C" perks_status perks_warmnet_predict(perks_warmnet *n, int32_t nimg, int32_t ny, int32_t nx, const double *k,
                                              const double *f, double *u, perks_stream stream) {
    if (!n) return PERKS_ERR_INVALID_ARG;
    if (nimg < 1 || ny < 1 || nx < 1 || !k || !f || !u) return fail(n->ctx, PERKS_ERR_INVALID_ARG, "warmnet_predict: bad arguments");
    perks_status rc = use_device(n->ctx);
    if (rc) return rc;
    if (ny % n->pool || nx % n->pool)
        return fail(n->ctx, PERKS_ERR_INVALID_ARG, "warmnet_predict: grid not divisible by the pool factor %d", n->pool);
    cudaStream_t s = (cudaStream_t)stream;
    const long long pixels = (long long)nimg * (ny / n->pool) * (nx / n->pool);
    rc = ensure_bufs(n, pixels);
    if (rc) return rc;
    rc = n->storage == PERKS_BF16 ? forward<__nv_bfloat16>(n, nimg, ny, nx, k, f, s) : forward<float>(n, nimg, ny, nx, k, f, s);
    if (rc) return rc;
    if (n->pool == 1) to_u_kernel<<<1024, 256, 0, s>>>(n->outb, n->out_scale, pixels, u);
    else upsample_kernel<<<1024, 256, 0, s>>>(n->outb, n->out_scale, ny, nx, n->pool, nimg, u);
    PERKS_CUDA(n->ctx, cudaGetLastError());
    return PERKS_OK;
}

extern "C" perks_status perks_warmnet_gradient(perks_warmnet *n, int32_t nimg, int32_t ny, int32_t nx, const double *k,
                                               const double *f, const double *u, float *grad_host, float *loss_host,
                                               perks_stream stream) {
    if (!n) return PERKS_ERR_INVALID_ARG;
    if (nimg < 1 || ny < 1 || nx < 1 || !k || !f || !u || ny % n->pool || nx % n->pool)
        return fail(n->ctx, PERKS_ERR_INVALID_ARG, "warmnet_gradient: bad arguments");
    perks_status rc = use_device(n->ctx);
    if (rc) return rc;
    cudaStream_t s = (cudaStream_t)stream;
    rc = loss_and_grad(n, nimg, ny, nx, k, f, u, s);
    if (rc) return rc;
    PERKS_CUDA(n->ctx, cudaStreamSynchronize(s));
    {
        DevError de{};
        PERKS_CUDA(n->ctx, cudaMemcpy(&de, n->err, sizeof(de), cudaMemcpyDeviceToHost));
        if (de.code) return fail(n->ctx, de.code, "warmnet: a tensor-core wait timed out (block %d)", de.block);
    }
    if (grad_host) PERKS_CUDA(n->ctx, cudaMemcpy(grad_host, n->grads, sizeof(float) * n->nparams, cudaMemcpyDeviceToHost));
    if (loss_host) PERKS_CUDA(n->ctx, cudaMemcpy(loss_host, n->loss, sizeof(float), cudaMemcpyDeviceToHost));
    return PERKS_OK;
}

extern "C" perks_status perks_warmnet_train_step(perks_warmnet *n, int32_t nimg, int32_t ny, int32_t nx,
                                                 const double *k, const double *f, const double *u, float lr,
                                                 perks_stream stream, float *loss_host) {
    if (!n) return PERKS_ERR_INVALID_ARG;
    if (nimg < 1 || ny < 1 || nx < 1 || !k || !f || !u || !(lr > 0.f) || ny % n->pool || nx % n->pool)
        return fail(n->ctx, PERKS_ERR_INVALID_ARG, "warmnet_train_step: bad arguments");
    perks_status rc = use_device(n->ctx);
    if (rc) return rc;
    cudaStream_t s = (cudaStream_t)stream;
    rc = loss_and_grad(n, nimg, ny, nx, k, f, u, s);
    if (rc) return rc;
    ++n->adam_t;
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = 1.f - std::pow(b1, (float)n->adam_t), c2 = 1.f - std::pow(b2, (float)n->adam_t);
    adam_kernel<<<(n->nparams + 255) / 256, 256, 0, s>>>(n->params, n->grads, n->m, n->v, n->nparams, lr, b1, b2,
                                                         1e-8f, c1, c2);
    PERKS_CUDA(n->ctx, cudaGetLastError());
    if (loss_host) {
        PERKS_CUDA(n->ctx, cudaMemcpyAsync(loss_host, n->loss, sizeof(float), cudaMemcpyDeviceToHost, s));
        PERKS_CUDA(n->ctx, cudaStreamSynchronize(s));
    }
    return PERKS_OK;
}

extern "C" perks_status perks_warmnet_fit(perks_warmnet *n, int32_t nimg, int32_t ny, int32_t nx, const double *k,
                                          const double *f, const double *u, int32_t batch, int32_t epochs, float lr,
                                          int32_t auto_scale, uint64_t seed, perks_stream stream, float *epoch_loss) {
    if (!n) return PERKS_ERR_INVALID_ARG;
    perks_context *ctx = n->ctx;
    if (nimg < 1 || ny < 1 || nx < 1 || !k || !f || !u || batch < 1 || epochs < 0 || !(lr > 0.f) ||
        ny % n->pool || nx % n->pool)
        return fail(ctx, PERKS_ERR_INVALID_ARG, "warmnet_fit: bad arguments");
    perks_status rc = use_device(ctx);
    if (rc) return rc;
    cudaStream_t s = (cudaStream_t)stream;
    const long long plane = (long long)ny * nx;
    if (auto_scale) {
        double *acc = nullptr;
        PERKS_CUDA(ctx, cudaMalloc(&acc, sizeof(double)));
        cudaError_t e = cudaMemsetAsync(acc, 0, sizeof(double), s);
        if (e == cudaSuccess) {
            sumsq_kernel<<<1024, 256, 0, s>>>(u, plane * nimg, acc);
            e = cudaGetLastError();
        }
        double h = 0.0;
        if (e == cudaSuccess) e = cudaMemcpyAsync(&h, acc, sizeof(double), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        cudaFree(acc);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "warmnet_fit: scale");
        const double rms = std::sqrt(h / (double)(plane * nimg));
        n->out_scale = rms > 0.0 ? (float)rms : 1.f;
    }
    const int nb = (nimg + batch - 1) / batch;
    std::vector<int> order(nb);
    Rng rng{seed};
    const float b1 = 0.9f, b2 = 0.999f;
    for (int ep = 0; ep < epochs; ++ep) {
        for (int i = 0; i < nb; ++i) order[i] = i;
        for (int i = nb - 1; i > 0; --i) std::swap(order[i], order[(int)(rng.next() % (uint64_t)(i + 1))]);
        double sum = 0.0;
        for (int bi = 0; bi < nb; ++bi) {
            const int i0 = order[bi] * batch, m = std::min(batch, nimg - i0);
            const long long o = (long long)i0 * plane;
            rc = loss_and_grad(n, m, ny, nx, k + o, f + o, u + o, s);
            if (rc) return rc;
            ++n->adam_t;
            const float c1 = 1.f - std::pow(b1, (float)n->adam_t), c2 = 1.f - std::pow(b2, (float)n->adam_t);
            adam_kernel<<<(n->nparams + 255) / 256, 256, 0, s>>>(n->params, n->grads, n->m, n->v, n->nparams, lr, b1,
                                                                 b2, 1e-8f, c1, c2);
            PERKS_CUDA(ctx, cudaGetLastError());
            if (epoch_loss) {
                float l = 0.f;
                PERKS_CUDA(ctx, cudaMemcpyAsync(&l, n->loss, sizeof(float), cudaMemcpyDeviceToHost, s));
                PERKS_CUDA(ctx, cudaStreamSynchronize(s));
                sum += (double)l * m;
            }
        }
        if (epoch_loss) epoch_loss[ep] = (float)(sum / nimg);
    }
    return PERKS_OK;
}

extern "C" perks_status perks_warmnet_set_tensor_cores(perks_warmnet *n, int32_t enable) {
    if (!n) return PERKS_ERR_INVALID_ARG;
    n->tensor_cores = enable != 0;
    return PERKS_OK;
}

extern "C" perks_status perks_warmnet_set_pool(perks_warmnet *n, int32_t factor) {
    if (!n) return PERKS_ERR_INVALID_ARG;
    if (factor < 1 || factor > 32) return fail(n->ctx, PERKS_ERR_INVALID_ARG, "warmnet_set_pool: factor in 1..32");
    n->pool = factor;
    return PERKS_OK;
}

extern "C" float perks_warmnet_get_scale(const perks_warmnet *n) { return n ? n->out_scale : 0.f; }
