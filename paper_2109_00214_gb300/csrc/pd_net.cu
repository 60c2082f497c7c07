// pd_net.cu -- the network of the learned Poisson warm start: inference,
// back-propagation of the mean squared error and Adam, all on the GPU.
//
// Six 3 x 3 convolutions over node grids (zero padding), channels 1 -> 32 ->
// 32 -> 32 -> 32 -> 32 -> 1, ReLU after the first five.  The four 32 -> 32
// layers, forward and back-propagation alike, are implicit GEMMs on the
// tensor cores (mma.sync m16n8k16, bfloat16 operands, float accumulators):
//   forward / input gradient: M = 16 nodes of a tile row, N = 32 output
//     channels, K = 9 taps x 32 input channels; a block stages an 8 x 16 node
//     tile with its halo and the layer's weights in shared memory.  The input
//     gradient is the same convolution over the output gradient with the
//     weights mirrored in the tap and transposed in the channels.
//   weight gradient: per tap, M = 32 output channels, N = 32 input channels,
//     K = the nodes, with one warp per tap; each block sums over the tiles it
//     visits and writes a partial that a second kernel adds up in a fixed
//     order (so the gradient does not depend on the launch).
// The 1 -> 32 and 32 -> 1 layers (1/32 of the arithmetic) run on the CUDA
// cores.  Storage: activations h_1..h_5 and the gradients with respect to
// a_1..a_5 in bfloat16 (node-major, 32 channels = 64 bytes per node), the
// input, output, targets and the output gradient in float, weights in
// bfloat16 for the layers and in float (master copies) for Adam.
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "pd.h"
#include "pd_net.h"

namespace pd {
namespace {

using bf16 = __nv_bfloat16;
constexpr int CH = 32;
constexpr int NP = PD_NET_NPARAMS;
// offsets of layer l's weights and biases in the parameter vector (layer 0:
// 288 weights + 32 biases; layers 1-4: 9216 + 32; layer 5: 288 + 1)
__host__ __device__ constexpr int off_w(int l) { return l == 0 ? 0 : (l < 5 ? 320 + (l - 1) * 9248 : 37312); }
__host__ __device__ constexpr int off_b(int l) { return l == 0 ? 288 : off_w(l) + (l < 5 ? 9216 : 288); }
static_assert(off_b(5) + 1 == PD_NET_NPARAMS, "parameter layout");
constexpr int TY = 8, TX = 16;       // node tile of the tensor-core kernels
constexpr int HP = 40;               // channel stride of a staged node (bf16): 80 bytes, conflict-free fragments
constexpr int GP = 24;               // node stride of the transposed tiles of the weight gradient
constexpr int MAX_PART_BLOCKS = 512;
constexpr int PART_STRIDE = 9 * CH * CH + CH;
constexpr int LOSS_BLOCKS = 256;

size_t al(size_t x) { return (x + 255) & ~(size_t)255; }

__device__ __forceinline__ int tap_dy(int tap) { return tap / 3 - 1; }
__device__ __forceinline__ int tap_dx(int tap) { return tap % 3 - 1; }

__device__ __forceinline__ void mma_bf16(float* c, uint32_t a0, uint32_t a1, uint32_t a2, uint32_t a3, uint32_t b0,
                                         uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

__device__ __forceinline__ uint32_t pack2(bf16 lo, bf16 hi) {
    return (uint32_t)__bfloat16_as_ushort(lo) | ((uint32_t)__bfloat16_as_ushort(hi) << 16);
}

__device__ __forceinline__ size_t node_index(const uint32_t* base, int b, int H, int W, int i, int j) {
    const size_t b0 = base ? (size_t)base[b] : (size_t)b * (size_t)H * (size_t)W;
    return b0 + (size_t)i * W + j;
}

// ---------------------------------------------------------------------------
// weights: float masters -> bfloat16 layer copies (wk: [tap][out][in]; wt:
// the input-gradient form, wt[tap'][in][out] = W[8 - tap'][out][in]) and
// bfloat16-rounded floats for the first and last layers
__global__ void k_prep_weights(const float* __restrict__ master, bf16* wk, bf16* wt, float* w1r, float* w6r) {
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q < 4 * 9 * CH * CH) {
        const int l = q / (9 * CH * CH), r = q % (9 * CH * CH);
        const int tap = r / (CH * CH), co = (r / CH) % CH, ci = r % CH;
        const bf16 v = __float2bfloat16_rn(master[off_w(l + 1) + r]);
        wk[q] = v;
        wt[l * 9 * CH * CH + ((8 - tap) * CH + ci) * CH + co] = v;
    }
    if (q < 9 * CH) {
        w1r[q] = __bfloat162float(__float2bfloat16_rn(master[off_w(0) + q]));
        w6r[q] = __bfloat162float(__float2bfloat16_rn(master[off_w(5) + q]));
    }
}

// ---------------------------------------------------------------------------
// layer 1 (1 -> 32): one thread per node
__global__ void __launch_bounds__(256) k_conv1(const float* __restrict__ x, bf16* __restrict__ h,
                                               const float* __restrict__ w1, const float* __restrict__ b1,
                                               const uint32_t* __restrict__ base, int B, int H, int W) {
    __shared__ float ws[9 * CH], bs[CH];
    for (int q = threadIdx.x; q < 9 * CH; q += blockDim.x) ws[q] = w1[q];
    if (threadIdx.x < CH) bs[threadIdx.x] = b1[threadIdx.x];
    __syncthreads();
    const long long n = (long long)H * W, total = n * B;
    for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < total;
         p += (long long)gridDim.x * blockDim.x) {
        const int b = (int)(p / n);
        const int k = (int)(p - (long long)b * n);
        const int i = k / W, j = k - i * W;
        float xv[9];
#pragma unroll
        for (int tap = 0; tap < 9; ++tap) {
            const int ii = i + tap_dy(tap), jj = j + tap_dx(tap);
            xv[tap] = (ii >= 0 && ii < H && jj >= 0 && jj < W) ? x[node_index(base, b, H, W, ii, jj)] : 0.0f;
        }
        uint32_t o[CH / 2];
#pragma unroll
        for (int c = 0; c < CH; c += 2) {
            float a0 = bs[c], a1 = bs[c + 1];
#pragma unroll
            for (int tap = 0; tap < 9; ++tap) {
                a0 += ws[tap * CH + c] * xv[tap];
                a1 += ws[tap * CH + c + 1] * xv[tap];
            }
            o[c / 2] = pack2(__float2bfloat16_rn(fmaxf(a0, 0.0f)), __float2bfloat16_rn(fmaxf(a1, 0.0f)));
        }
        uint4* dst = (uint4*)(h + node_index(base, b, H, W, i, j) * CH);
#pragma unroll
        for (int q = 0; q < 4; ++q) dst[q] = make_uint4(o[4 * q], o[4 * q + 1], o[4 * q + 2], o[4 * q + 3]);
    }
}

// ---------------------------------------------------------------------------
// 32 -> 32 convolution on the tensor cores.  MODE 0: out = relu(conv + bias);
// MODE 1: out = conv where mask > 0, else 0 (input gradient through a ReLU).
// Block: 8 warps, an 8 x 16 node tile (warp w: tile row w), grid (tiles
// along j, tiles along i, samples).
template <int MODE>
__global__ void __launch_bounds__(256) k_conv32(const bf16* __restrict__ in, bf16* __restrict__ out,
                                                const bf16* __restrict__ w, const float* __restrict__ bias,
                                                const bf16* __restrict__ mask, const uint32_t* __restrict__ base,
                                                int H, int W) {
    __shared__ __align__(16) bf16 xs[(TY + 2) * (TX + 2) * HP];
    __shared__ __align__(16) bf16 ws[9 * CH * HP];
    const int b = blockIdx.z;
    const int i0 = blockIdx.y * TY, j0 = blockIdx.x * TX;
    for (int q = threadIdx.x; q < 9 * CH * 4; q += blockDim.x) {
        const int row = q >> 2, part = q & 3;
        *(uint4*)&ws[row * HP + part * 8] = ((const uint4*)w)[q];
    }
    for (int q = threadIdx.x; q < (TY + 2) * (TX + 2) * 4; q += blockDim.x) {
        const int nd = q >> 2, part = q & 3;
        const int hi = nd / (TX + 2), hj = nd - hi * (TX + 2);
        const int gi = i0 + hi - 1, gj = j0 + hj - 1;
        uint4 v = make_uint4(0u, 0u, 0u, 0u);
        if (gi >= 0 && gi < H && gj >= 0 && gj < W) v = ((const uint4*)(in + node_index(base, b, H, W, gi, gj) * CH))[part];
        *(uint4*)&xs[nd * HP + part * 8] = v;
    }
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
    float acc[4][4];
#pragma unroll
    for (int nt = 0; nt < 4; ++nt)
#pragma unroll
        for (int e = 0; e < 4; ++e) acc[nt][e] = 0.0f;
#pragma unroll 1
    for (int tap = 0; tap < 9; ++tap) {
        const bf16* xr = xs + ((warp + tap_dy(tap) + 1) * (TX + 2) + tap_dx(tap) + 1) * HP;
#pragma unroll
        for (int kh = 0; kh < 2; ++kh) {
            const int c0 = kh * 16 + 2 * t;
            const uint32_t a0 = *(const uint32_t*)(xr + g * HP + c0);
            const uint32_t a1 = *(const uint32_t*)(xr + (g + 8) * HP + c0);
            const uint32_t a2 = *(const uint32_t*)(xr + g * HP + c0 + 8);
            const uint32_t a3 = *(const uint32_t*)(xr + (g + 8) * HP + c0 + 8);
#pragma unroll
            for (int nt = 0; nt < 4; ++nt) {
                const bf16* wr = ws + (tap * CH + nt * 8 + g) * HP + c0;
                mma_bf16(acc[nt], a0, a1, a2, a3, *(const uint32_t*)wr, *(const uint32_t*)(wr + 8));
            }
        }
    }
    const int oi = i0 + warp;
    if (oi >= H) return;
#pragma unroll
    for (int half = 0; half < 2; ++half) {
        const int oj = j0 + g + 8 * half;
        if (oj >= W) continue;
        const size_t nd = node_index(base, b, H, W, oi, oj);
#pragma unroll
        for (int nt = 0; nt < 4; ++nt) {
            const int c = nt * 8 + 2 * t;
            float v0 = acc[nt][2 * half], v1 = acc[nt][2 * half + 1];
            if (MODE == 0) {
                v0 = fmaxf(v0 + bias[c], 0.0f);
                v1 = fmaxf(v1 + bias[c + 1], 0.0f);
            } else {
                const __nv_bfloat162 m = *(const __nv_bfloat162*)(mask + nd * CH + c);
                if (!(__bfloat162float(m.x) > 0.0f)) v0 = 0.0f;
                if (!(__bfloat162float(m.y) > 0.0f)) v1 = 0.0f;
            }
            *(__nv_bfloat162*)(out + nd * CH + c) = __floats2bfloat162_rn(v0, v1);
        }
    }
}

// ---------------------------------------------------------------------------
// layer 6 (32 -> 1): one thread per node
__global__ void __launch_bounds__(256) k_conv6(const bf16* __restrict__ h, float* __restrict__ y,
                                               const float* __restrict__ w6, const float* __restrict__ b6,
                                               const uint32_t* __restrict__ base, int B, int H, int W) {
    __shared__ float ws[9 * CH];
    for (int q = threadIdx.x; q < 9 * CH; q += blockDim.x) ws[q] = w6[q];
    __syncthreads();
    const float bias = b6[0];
    const long long n = (long long)H * W, total = n * B;
    for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < total;
         p += (long long)gridDim.x * blockDim.x) {
        const int b = (int)(p / n);
        const int k = (int)(p - (long long)b * n);
        const int i = k / W, j = k - i * W;
        float acc = bias;
        for (int tap = 0; tap < 9; ++tap) {
            const int ii = i + tap_dy(tap), jj = j + tap_dx(tap);
            if (ii < 0 || ii >= H || jj < 0 || jj >= W) continue;
            const uint4* src = (const uint4*)(h + node_index(base, b, H, W, ii, jj) * CH);
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const uint4 v = src[q];
                const uint32_t u[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    const int c = q * 8 + e * 2;
                    acc += ws[tap * CH + c] * __uint_as_float(u[e] << 16);
                    acc += ws[tap * CH + c + 1] * __uint_as_float(u[e] & 0xFFFF0000u);
                }
            }
        }
        y[node_index(base, b, H, W, i, j)] = acc;
    }
}

// ---------------------------------------------------------------------------
// loss: g6 = 2 (y - t) / N and per-block partial sums of (y - t)^2
__global__ void __launch_bounds__(256) k_loss(const float* __restrict__ y, const float* __restrict__ t, float* g6,
                                              double* part, long long n) {
    double acc = 0.0;
    const float s = (float)(2.0 / (double)n);
    for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < n;
         p += (long long)gridDim.x * blockDim.x) {
        const float d = y[p] - t[p];
        g6[p] = s * d;
        acc += (double)d * (double)d;
    }
    __shared__ double red[256];
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = red[0];
}

// residual loss of a start on an r-z grid (dz = dr): the unit finite-volume
// coefficients of radial node j of W, and (S v)_ij on an interior row with
// rows 0 and H - 1 of v read as zero (Dirichlet)
__device__ __forceinline__ void rz_coeffs(int j, int W, float& ap, float& am, float& w) {
    const int nr = W - 1;
    ap = j < nr ? (float)j + 0.5f : 0.0f;
    am = j > 0 ? (float)j - 0.5f : 0.0f;
    w = j == 0 ? 0.125f : (j == nr ? 0.5f * (float)nr - 0.125f : (float)j);
}
__device__ __forceinline__ float rz_apply(const float* __restrict__ v, size_t k, int H, int W, int i, int j) {
    float ap, am, w;
    rz_coeffs(j, W, ap, am, w);
    float s = (ap + am + 2.0f * w) * v[k];
    if (j + 1 < W) s -= ap * v[k + 1];
    if (j > 0) s -= am * v[k - 1];
    if (i + 1 < H - 1) s -= w * v[k + W];
    if (i - 1 > 0) s -= w * v[k - W];
    return s;
}

// r = w x - S y on the interior rows (0 on the electrode rows) and
// per-block partial sums of r^2
__global__ void __launch_bounds__(256) k_rz_resid(const float* __restrict__ x, const float* __restrict__ y,
                                                  float* __restrict__ r, double* part, int B, int H, int W) {
    const long long n = (long long)B * H * W;
    double acc = 0.0;
    for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < n;
         p += (long long)gridDim.x * blockDim.x) {
        const int q = (int)(p % ((long long)H * W)), i = q / W, j = q - i * W;
        if (i == 0 || i == H - 1) {
            r[p] = 0.0f;
            continue;
        }
        float ap, am, w;
        rz_coeffs(j, W, ap, am, w);
        const float v = w * x[p] - rz_apply(y, (size_t)p, H, W, i, j);
        r[p] = v;
        acc += (double)v * (double)v;
    }
    __shared__ double red[256];
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = red[0];
}

// g = scale S r on the interior rows, 0 on the electrode rows (S is
// symmetric, so this is scale S^T r)
__global__ void __launch_bounds__(256) k_rz_resid_grad(const float* __restrict__ r, float* __restrict__ g, float scale,
                                                       int B, int H, int W) {
    const long long n = (long long)B * H * W;
    for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < n;
         p += (long long)gridDim.x * blockDim.x) {
        const int q = (int)(p % ((long long)H * W)), i = q / W, j = q - i * W;
        g[p] = (i == 0 || i == H - 1) ? 0.0f : scale * rz_apply(r, (size_t)p, H, W, i, j);
    }
}

__global__ void k_loss_sum(const double* part, int n, double inv_count, double* out) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        double s = 0.0;
        for (int q = 0; q < n; ++q) s += part[q];
        *out = s * inv_count;
    }
}

// gradient with respect to a_5: (sum_tap w6[tap][c] g6[p - tap]) where h5 > 0
__global__ void __launch_bounds__(256) k_conv6_bwd(const float* __restrict__ g6, const bf16* __restrict__ h5,
                                                   bf16* __restrict__ g5, const float* __restrict__ w6, int B, int H,
                                                   int W) {
    __shared__ float ws[9 * CH];
    for (int q = threadIdx.x; q < 9 * CH; q += blockDim.x) ws[q] = w6[q];
    __syncthreads();
    const long long n = (long long)H * W, total = n * B;
    for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < total;
         p += (long long)gridDim.x * blockDim.x) {
        const int b = (int)(p / n);
        const int k = (int)(p - (long long)b * n);
        const int i = k / W, j = k - i * W;
        float gv[9];
#pragma unroll
        for (int tap = 0; tap < 9; ++tap) {
            const int ii = i - tap_dy(tap), jj = j - tap_dx(tap);
            gv[tap] = (ii >= 0 && ii < H && jj >= 0 && jj < W) ? g6[(size_t)b * n + (size_t)ii * W + jj] : 0.0f;
        }
        const uint4* hm = (const uint4*)(h5 + (size_t)p * CH);
        uint4* dst = (uint4*)(g5 + (size_t)p * CH);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const uint4 mv = hm[q];
            const uint32_t mu[4] = {mv.x, mv.y, mv.z, mv.w};
            uint32_t o[4];
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const int c = q * 8 + e * 2;
                float a0 = 0.0f, a1 = 0.0f;
#pragma unroll
                for (int tap = 0; tap < 9; ++tap) {
                    a0 += ws[tap * CH + c] * gv[tap];
                    a1 += ws[tap * CH + c + 1] * gv[tap];
                }
                if (!(__uint_as_float(mu[e] << 16) > 0.0f)) a0 = 0.0f;
                if (!(__uint_as_float(mu[e] & 0xFFFF0000u) > 0.0f)) a1 = 0.0f;
                o[e] = pack2(__float2bfloat16_rn(a0), __float2bfloat16_rn(a1));
            }
            dst[q] = make_uint4(o[0], o[1], o[2], o[3]);
        }
    }
}

// ---------------------------------------------------------------------------
// weight gradients of the first and last layers (CUDA cores), over the same
// 8 x 16 node tiles staged in shared memory: thread (tap, c) < 288 of a
// 320-thread block sums over the tiles the block visits; the remaining
// threads sum the bias gradients.  Partials: [block][288 + biases].
__global__ void __launch_bounds__(320) k_wgrad1(const float* __restrict__ x, const bf16* __restrict__ g1,
                                                float* part, int B, int H, int W) {
    __shared__ float gsm[TY * TX][CH + 1];
    __shared__ float xsm[(TY + 2) * (TX + 2)];
    const int tid = threadIdx.x;
    const int tap = tid / CH, co = tid % CH;
    const int dy = tap < 9 ? tap_dy(tap) : 0, dx = tap < 9 ? tap_dx(tap) : 0;
    const int tj = (W + TX - 1) / TX, ti = (H + TY - 1) / TY;
    const long long ntiles = (long long)B * tj * ti, n = (long long)H * W;
    float acc = 0.0f;
    for (long long tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const int b = (int)(tile / ((long long)tj * ti));
        const int r = (int)(tile - (long long)b * tj * ti);
        const int i0 = (r / tj) * TY, j0 = (r % tj) * TX;
        __syncthreads();
        for (int q = tid; q < TY * TX * CH; q += blockDim.x) {
            const int nd = q / CH, c = q % CH;
            const int gi = i0 + nd / TX, gj = j0 + nd % TX;
            gsm[nd][c] = (gi < H && gj < W) ? __bfloat162float(g1[((size_t)b * n + (size_t)gi * W + gj) * CH + c]) : 0.0f;
        }
        for (int q = tid; q < (TY + 2) * (TX + 2); q += blockDim.x) {
            const int gi = i0 + q / (TX + 2) - 1, gj = j0 + q % (TX + 2) - 1;
            xsm[q] = (gi >= 0 && gi < H && gj >= 0 && gj < W) ? x[(size_t)b * n + (size_t)gi * W + gj] : 0.0f;
        }
        __syncthreads();
        if (tid < 9 * CH) {
            for (int nd = 0; nd < TY * TX; ++nd)
                acc += gsm[nd][co] * xsm[(nd / TX + dy + 1) * (TX + 2) + nd % TX + dx + 1];
        } else {
            for (int nd = 0; nd < TY * TX; ++nd) acc += gsm[nd][tid - 9 * CH];
        }
    }
    part[(size_t)blockIdx.x * (9 * CH + CH) + tid] = acc;
}

__global__ void __launch_bounds__(320) k_wgrad6(const float* __restrict__ g6, const bf16* __restrict__ h5,
                                                float* part, int B, int H, int W) {
    __shared__ float gsm[TY * TX];
    __shared__ float hsm[(TY + 2) * (TX + 2)][CH + 1];
    const int tid = threadIdx.x;
    const int tap = tid / CH, ci = tid % CH;
    const int dy = tap < 9 ? tap_dy(tap) : 0, dx = tap < 9 ? tap_dx(tap) : 0;
    const int tj = (W + TX - 1) / TX, ti = (H + TY - 1) / TY;
    const long long ntiles = (long long)B * tj * ti, n = (long long)H * W;
    float acc = 0.0f;
    for (long long tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const int b = (int)(tile / ((long long)tj * ti));
        const int r = (int)(tile - (long long)b * tj * ti);
        const int i0 = (r / tj) * TY, j0 = (r % tj) * TX;
        __syncthreads();
        for (int q = tid; q < TY * TX; q += blockDim.x) {
            const int gi = i0 + q / TX, gj = j0 + q % TX;
            gsm[q] = (gi < H && gj < W) ? g6[(size_t)b * n + (size_t)gi * W + gj] : 0.0f;
        }
        for (int q = tid; q < (TY + 2) * (TX + 2) * CH; q += blockDim.x) {
            const int nd = q / CH, c = q % CH;
            const int gi = i0 + nd / (TX + 2) - 1, gj = j0 + nd % (TX + 2) - 1;
            hsm[nd][c] = (gi >= 0 && gi < H && gj >= 0 && gj < W)
                             ? __bfloat162float(h5[((size_t)b * n + (size_t)gi * W + gj) * CH + c])
                             : 0.0f;
        }
        __syncthreads();
        if (tid < 9 * CH) {
            for (int nd = 0; nd < TY * TX; ++nd)
                acc += gsm[nd] * hsm[(nd / TX + dy + 1) * (TX + 2) + nd % TX + dx + 1][ci];
        } else if (tid == 9 * CH) {
            for (int nd = 0; nd < TY * TX; ++nd) acc += gsm[nd];
        }
    }
    if (tid <= 9 * CH) part[(size_t)blockIdx.x * (9 * CH + 1) + tid] = acc;
}

// weight gradient of a 32 -> 32 layer on the tensor cores: warp = tap.
// Tiles are staged transposed (channel-major rows of 16 nodes) so that the
// node index is the contiguous GEMM k dimension of both operands.
__global__ void __launch_bounds__(288) k_wgrad32(const bf16* __restrict__ h, const bf16* __restrict__ g,
                                                 float* part, int B, int H, int W) {
    __shared__ __align__(16) bf16 gs[TY * CH * GP];          // [row][co][col]
    __shared__ __align__(16) bf16 hs[(TY + 2) * CH * GP];    // [halo row][ci][halo col]
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, gq = lane >> 2, t = lane & 3;
    const int dy = tap_dy(warp), dx = tap_dx(warp);
    float acc[2][4][4];
#pragma unroll
    for (int mt = 0; mt < 2; ++mt)
#pragma unroll
        for (int nt = 0; nt < 4; ++nt)
#pragma unroll
            for (int e = 0; e < 4; ++e) acc[mt][nt][e] = 0.0f;
    float bacc = 0.0f;
    const int tj = (W + TX - 1) / TX, ti = (H + TY - 1) / TY;
    const long long ntiles = (long long)B * tj * ti;
    const long long n = (long long)H * W;
    for (long long tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const int b = (int)(tile / ((long long)tj * ti));
        const int r = (int)(tile - (long long)b * tj * ti);
        const int i0 = (r / tj) * TY, j0 = (r % tj) * TX;
        __syncthreads();
        for (int q = threadIdx.x; q < TY * TX * 4; q += blockDim.x) {
            const int nd = q >> 2, part4 = q & 3;
            const int ri = nd / TX, rj = nd - ri * TX;
            const int gi = i0 + ri, gj = j0 + rj;
            uint4 v = make_uint4(0u, 0u, 0u, 0u);
            if (gi < H && gj < W) v = ((const uint4*)(g + ((size_t)b * n + (size_t)gi * W + gj) * CH))[part4];
            const bf16* e = (const bf16*)&v;
#pragma unroll
            for (int k = 0; k < 8; ++k) gs[(ri * CH + part4 * 8 + k) * GP + rj] = e[k];
        }
        for (int q = threadIdx.x; q < (TY + 2) * (TX + 2) * 4; q += blockDim.x) {
            const int nd = q >> 2, part4 = q & 3;
            const int hi = nd / (TX + 2), hj = nd - hi * (TX + 2);
            const int gi = i0 + hi - 1, gj = j0 + hj - 1;
            uint4 v = make_uint4(0u, 0u, 0u, 0u);
            if (gi >= 0 && gi < H && gj >= 0 && gj < W)
                v = ((const uint4*)(h + ((size_t)b * n + (size_t)gi * W + gj) * CH))[part4];
            const bf16* e = (const bf16*)&v;
#pragma unroll
            for (int k = 0; k < 8; ++k) hs[(hi * CH + part4 * 8 + k) * GP + hj] = e[k];
        }
        __syncthreads();
#pragma unroll 1
        for (int ri = 0; ri < TY; ++ri) {
            uint32_t a[2][4];
#pragma unroll
            for (int mt = 0; mt < 2; ++mt) {
                const bf16* gr = gs + (ri * CH + mt * 16 + gq) * GP + 2 * t;
                a[mt][0] = *(const uint32_t*)gr;
                a[mt][1] = *(const uint32_t*)(gr + 8 * GP);
                a[mt][2] = *(const uint32_t*)(gr + 8);
                a[mt][3] = *(const uint32_t*)(gr + 8 * GP + 8);
            }
#pragma unroll
            for (int nt = 0; nt < 4; ++nt) {
                const bf16* hr = hs + ((ri + dy + 1) * CH + nt * 8 + gq) * GP + dx + 1;
                const uint32_t b0 = pack2(hr[2 * t], hr[2 * t + 1]);
                const uint32_t b1 = pack2(hr[2 * t + 8], hr[2 * t + 9]);
#pragma unroll
                for (int mt = 0; mt < 2; ++mt) mma_bf16(acc[mt][nt], a[mt][0], a[mt][1], a[mt][2], a[mt][3], b0, b1);
            }
        }
        if (threadIdx.x < CH)
            for (int ri = 0; ri < TY; ++ri)
                for (int rj = 0; rj < TX; ++rj) bacc += __bfloat162float(gs[(ri * CH + threadIdx.x) * GP + rj]);
    }
    float* P = part + (size_t)blockIdx.x * PART_STRIDE;
#pragma unroll
    for (int mt = 0; mt < 2; ++mt)
#pragma unroll
        for (int nt = 0; nt < 4; ++nt) {
            const int co = mt * 16 + gq, ci = nt * 8 + 2 * t;
            P[(warp * CH + co) * CH + ci] = acc[mt][nt][0];
            P[(warp * CH + co) * CH + ci + 1] = acc[mt][nt][1];
            P[(warp * CH + co + 8) * CH + ci] = acc[mt][nt][2];
            P[(warp * CH + co + 8) * CH + ci + 1] = acc[mt][nt][3];
        }
    if (threadIdx.x < CH) P[9 * CH * CH + threadIdx.x] = bacc;
}

// out[k] = sum over blocks c (in order) of part[c * stride + k], k < count
__global__ void k_reduce(const float* __restrict__ part, int nblocks, int stride, int count, float* out) {
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < count; k += gridDim.x * blockDim.x) {
        float s = 0.0f;
        for (int c = 0; c < nblocks; ++c) s += part[(size_t)c * stride + k];
        out[k] = s;
    }
}

__global__ void k_adam(float* w, float* m, float* v, const float* __restrict__ g, float lr, float b1, float b2,
                       float eps, float c1, float c2) {
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= NP) return;
    const float gq = g[q];
    const float mq = b1 * m[q] + (1.0f - b1) * gq;
    const float vq = b2 * v[q] + (1.0f - b2) * gq * gq;
    m[q] = mq;
    v[q] = vq;
    w[q] -= lr * (mq / c1) / (sqrtf(vq / c2) + eps);
}

}  // namespace
}  // namespace pd

using namespace pd;

struct pd_net {
    int64_t max_nodes;
    cudaStream_t stream;
    int sms;
    float *master, *m, *v, *grad;
    bf16 *wk, *wt;
    float *w1r, *w6r;
    bf16* h[5];
    bf16* g[5];
    float *g6, *ybuf;
    float* part;
    double *lpart, *lsum;
    int64_t adam_k;
    bool have_grad;
    std::string err;
};

namespace {

struct NetLayout {
    size_t master, m, v, grad, wk, wt, w1r, w6r, h[5], g[5], g6, ybuf, part, lpart, lsum, total;
};

NetLayout net_layout(int64_t max_nodes) {
    NetLayout L;
    size_t o = 0;
    auto take = [&](size_t b) {
        const size_t r = o;
        o += al(b);
        return r;
    };
    L.master = take(NP * 4);
    L.m = take(NP * 4);
    L.v = take(NP * 4);
    L.grad = take(NP * 4);
    L.wk = take(4 * 9 * CH * CH * 2);
    L.wt = take(4 * 9 * CH * CH * 2);
    L.w1r = take(9 * CH * 4);
    L.w6r = take(9 * CH * 4);
    for (int l = 0; l < 5; ++l) L.h[l] = take((size_t)max_nodes * CH * 2);
    for (int l = 0; l < 5; ++l) L.g[l] = take((size_t)max_nodes * CH * 2);
    L.g6 = take((size_t)max_nodes * 4);
    L.ybuf = take((size_t)max_nodes * 4);
    L.part = take((size_t)MAX_PART_BLOCKS * PART_STRIDE * 4);
    L.lpart = take(LOSS_BLOCKS * 8);
    L.lsum = take(8);
    L.total = o;
    return L;
}

int part_blocks(const pd_net* net) { return std::min(MAX_PART_BLOCKS, 2 * net->sms); }
int elem_blocks(const pd_net* net, long long n) {
    const long long b = (n + 255) / 256;
    return (int)std::max(1LL, std::min(b, (long long)net->sms * 16));
}

pd_status net_fail(pd_net* net, pd_status code, const std::string& msg) {
    if (net) net->err = msg;
    return code;
}

bool shape_ok(const pd_net* net, int B, int H, int W) {
    return B >= 1 && H >= 1 && W >= 1 && (int64_t)B * H * W <= net->max_nodes;
}

void forward_layers(pd_net* net, const float* x, float* y, int B, int H, int W, const uint32_t* base,
                    cudaStream_t s) {
    const long long total = (long long)B * H * W;
    const float* P = net->master;
    k_conv1<<<elem_blocks(net, total), 256, 0, s>>>(x, net->h[0], net->w1r, P + off_b(0), base, B, H, W);
    const dim3 grid((W + TX - 1) / TX, (H + TY - 1) / TY, B);
    for (int l = 1; l <= 4; ++l)
        k_conv32<0><<<grid, 256, 0, s>>>(net->h[l - 1], net->h[l], net->wk + (size_t)(l - 1) * 9 * CH * CH,
                                         P + off_b(l), nullptr, base, H, W);
    k_conv6<<<elem_blocks(net, total), 256, 0, s>>>(net->h[4], y, net->w6r, P + off_b(5), base, B, H, W);
}

pd_status upload_weights(pd_net* net) {
    k_prep_weights<<<(4 * 9 * CH * CH + 255) / 256, 256, 0, net->stream>>>(net->master, net->wk, net->wt, net->w1r,
                                                                          net->w6r);
    const cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? PD_OK : net_fail(net, PD_ERR_CUDA, cudaGetErrorString(e));
}

}  // namespace

namespace pd {
int net_forward_at(pd_net* net, const float* x, float* y, int B, int H, int W, const uint32_t* base,
                   int64_t node_span, cudaStream_t stream) {
    if (!net || node_span > net->max_nodes) return 1;
    forward_layers(net, x, y, B, H, W, base, stream);
    return cudaGetLastError() == cudaSuccess ? 0 : 1;
}
int64_t net_max_nodes(const pd_net* net) { return net ? net->max_nodes : 0; }
}  // namespace pd

extern "C" {

pd_status pd_net_workspace_size(int64_t max_nodes, size_t* bytes) {
    if (!bytes || max_nodes < 1 || max_nodes > (int64_t)1 << 31) return PD_ERR_ARG;
    *bytes = net_layout(max_nodes).total;
    return PD_OK;
}

pd_status pd_net_create(int64_t max_nodes, void* ws, size_t bytes, void* stream, pd_net** out) {
    if (!out) return PD_ERR_ARG;
    *out = nullptr;
    if (max_nodes < 1 || max_nodes > (int64_t)1 << 31 || !ws || ((uintptr_t)ws & 255)) return PD_ERR_ARG;
    const NetLayout L = net_layout(max_nodes);
    if (bytes < L.total) return PD_ERR_ARG;
    pd_net* net = new (std::nothrow) pd_net();
    if (!net) return PD_ERR_ARG;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&net->sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        delete net;
        return PD_ERR_CUDA;
    }
    char* w = (char*)ws;
    net->max_nodes = max_nodes;
    net->stream = (cudaStream_t)stream;
    net->master = (float*)(w + L.master);
    net->m = (float*)(w + L.m);
    net->v = (float*)(w + L.v);
    net->grad = (float*)(w + L.grad);
    net->wk = (bf16*)(w + L.wk);
    net->wt = (bf16*)(w + L.wt);
    net->w1r = (float*)(w + L.w1r);
    net->w6r = (float*)(w + L.w6r);
    for (int l = 0; l < 5; ++l) {
        net->h[l] = (bf16*)(w + L.h[l]);
        net->g[l] = (bf16*)(w + L.g[l]);
    }
    net->g6 = (float*)(w + L.g6);
    net->ybuf = (float*)(w + L.ybuf);
    net->part = (float*)(w + L.part);
    net->lpart = (double*)(w + L.lpart);
    net->lsum = (double*)(w + L.lsum);
    net->adam_k = 0;
    net->have_grad = false;
    if (cudaMemsetAsync(w, 0, L.g6, net->stream) != cudaSuccess || upload_weights(net) != PD_OK ||
        cudaStreamSynchronize(net->stream) != cudaSuccess) {
        delete net;
        return PD_ERR_CUDA;
    }
    *out = net;
    return PD_OK;
}

void pd_net_destroy(pd_net* net) {
    if (!net) return;
    cudaStreamSynchronize(net->stream);
    delete net;
}

pd_status pd_net_set_params(pd_net* net, const float* params) {
    if (!net || !params) return PD_ERR_ARG;
    if (cudaMemcpyAsync(net->master, params, NP * 4, cudaMemcpyHostToDevice, net->stream) != cudaSuccess ||
        cudaMemsetAsync(net->m, 0, NP * 4, net->stream) != cudaSuccess ||
        cudaMemsetAsync(net->v, 0, NP * 4, net->stream) != cudaSuccess)
        return net_fail(net, PD_ERR_CUDA, "parameter upload failed");
    net->adam_k = 0;
    net->have_grad = false;
    const pd_status r = upload_weights(net);
    if (r != PD_OK) return r;
    return cudaStreamSynchronize(net->stream) == cudaSuccess ? PD_OK : net_fail(net, PD_ERR_CUDA, "sync failed");
}

pd_status pd_net_get_params(pd_net* net, float* params) {
    if (!net || !params) return PD_ERR_ARG;
    if (cudaMemcpyAsync(params, net->master, NP * 4, cudaMemcpyDeviceToHost, net->stream) != cudaSuccess ||
        cudaStreamSynchronize(net->stream) != cudaSuccess)
        return net_fail(net, PD_ERR_CUDA, "parameter download failed");
    return PD_OK;
}

pd_status pd_net_forward(pd_net* net, const float* x, int B, int H, int W, float* y) {
    if (!net || !x || !y) return PD_ERR_ARG;
    if (!shape_ok(net, B, H, W)) return net_fail(net, PD_ERR_ARG, "batch exceeds the network's node capacity");
    forward_layers(net, x, y, B, H, W, nullptr, net->stream);
    const cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? PD_OK : net_fail(net, PD_ERR_CUDA, cudaGetErrorString(e));
}

}  // extern "C"

namespace {

// back-propagation of the output gradient g6 (B H W floats) to the
// parameter gradient, and the loss and gradient out to the host if asked
pd_status backprop(pd_net* net, const float* x, const float* g6, int B, int H, int W, double* loss, float* grads) {
    cudaStream_t s = net->stream;
    const long long total = (long long)B * H * W;
    const int pb = part_blocks(net);
    const int eb = elem_blocks(net, total);
    // layer 6
    k_wgrad6<<<pb, 320, 0, s>>>(g6, net->h[4], net->part, B, H, W);
    k_reduce<<<2, 160, 0, s>>>(net->part, pb, 9 * CH + 1, 9 * CH + 1, net->grad + off_w(5));
    k_conv6_bwd<<<eb, 256, 0, s>>>(g6, net->h[4], net->g[4], net->w6r, B, H, W);
    // layers 5 .. 2
    const dim3 grid((W + TX - 1) / TX, (H + TY - 1) / TY, B);
    for (int l = 4; l >= 1; --l) {
        k_wgrad32<<<pb, 288, 0, s>>>(net->h[l - 1], net->g[l], net->part, B, H, W);
        // weights then biases: both contiguous in the parameter vector
        k_reduce<<<(PART_STRIDE + 255) / 256, 256, 0, s>>>(net->part, pb, PART_STRIDE, PART_STRIDE,
                                                          net->grad + off_w(l));
        k_conv32<1><<<grid, 256, 0, s>>>(net->g[l], net->g[l - 1], net->wt + (size_t)(l - 1) * 9 * CH * CH,
                                         nullptr, net->h[l - 1], nullptr, H, W);
    }
    // layer 1
    k_wgrad1<<<pb, 320, 0, s>>>(x, net->g[0], net->part, B, H, W);
    k_reduce<<<2, 160, 0, s>>>(net->part, pb, 9 * CH + CH, 9 * CH + CH, net->grad + off_w(0));
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return net_fail(net, PD_ERR_CUDA, cudaGetErrorString(e));
    net->have_grad = true;
    if (loss) e = cudaMemcpyAsync(loss, net->lsum, 8, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess && grads) e = cudaMemcpyAsync(grads, net->grad, NP * 4, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess && (loss || grads)) e = cudaStreamSynchronize(s);
    return e == cudaSuccess ? PD_OK : net_fail(net, PD_ERR_CUDA, cudaGetErrorString(e));
}

}  // namespace

extern "C" {

pd_status pd_net_loss_grad(pd_net* net, const float* x, const float* t, int B, int H, int W, double* loss,
                           float* grads) {
    if (!net || !x || !t) return PD_ERR_ARG;
    if (!shape_ok(net, B, H, W)) return net_fail(net, PD_ERR_ARG, "batch exceeds the network's node capacity");
    cudaStream_t s = net->stream;
    const long long total = (long long)B * H * W;
    forward_layers(net, x, net->ybuf, B, H, W, nullptr, s);
    const int lb = (int)std::min<long long>(LOSS_BLOCKS, (total + 255) / 256);
    k_loss<<<lb, 256, 0, s>>>(net->ybuf, t, net->g6, net->lpart, total);
    k_loss_sum<<<1, 32, 0, s>>>(net->lpart, lb, 1.0 / (double)total, net->lsum);
    return backprop(net, x, net->g6, B, H, W, loss, grads);
}

pd_status pd_net_loss_grad_rz(pd_net* net, const float* x, int B, int H, int W, double* loss, float* grads) {
    if (!net || !x) return PD_ERR_ARG;
    if (!shape_ok(net, B, H, W) || H < 3 || W < 2)
        return net_fail(net, PD_ERR_ARG, "batch exceeds the network's node capacity, or a grid below 3 x 2 nodes");
    cudaStream_t s = net->stream;
    const long long total = (long long)B * H * W, n_int = (long long)B * (H - 2) * W;
    forward_layers(net, x, net->ybuf, B, H, W, nullptr, s);
    const int lb = (int)std::min<long long>(LOSS_BLOCKS, (total + 255) / 256);
    // r into g6, then dL/dy = -(2 / N) S r into ybuf (y is not needed after r)
    k_rz_resid<<<lb, 256, 0, s>>>(x, net->ybuf, net->g6, net->lpart, B, H, W);
    k_loss_sum<<<1, 32, 0, s>>>(net->lpart, lb, 1.0 / (double)n_int, net->lsum);
    k_rz_resid_grad<<<elem_blocks(net, total), 256, 0, s>>>(net->g6, net->ybuf, (float)(-2.0 / (double)n_int), B, H,
                                                           W);
    return backprop(net, x, net->ybuf, B, H, W, loss, grads);
}

pd_status pd_net_adam(pd_net* net, float lr, float b1, float b2, float eps) {
    if (!net) return PD_ERR_ARG;
    if (!net->have_grad) return net_fail(net, PD_ERR_STATE, "no gradient: call pd_net_loss_grad first");
    if (!(lr > 0) || !(b1 >= 0 && b1 < 1) || !(b2 >= 0 && b2 < 1) || !(eps >= 0))
        return net_fail(net, PD_ERR_ARG, "bad Adam hyper-parameters");
    net->adam_k += 1;
    const float c1 = (float)(1.0 - std::pow((double)b1, (double)net->adam_k));
    const float c2 = (float)(1.0 - std::pow((double)b2, (double)net->adam_k));
    k_adam<<<(NP + 255) / 256, 256, 0, net->stream>>>(net->master, net->m, net->v, net->grad, lr, b1, b2, eps, c1,
                                                      c2);
    return upload_weights(net);
}

}  // extern "C"
