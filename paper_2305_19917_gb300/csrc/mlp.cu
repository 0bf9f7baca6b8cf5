// Cost-model network: a 3 x 64 GELU multilayer perceptron mapping plan
// features to log execution time.  It stands in for the paper's analytical
// performance models (Section V: Comp(i) of the recursive, iterative and
// blocked models, and the refinement stop rule), learned from timings that
// the autotuner measures on this GPU.  Hand-written forward, backward, loss
// and Adam kernels (FP32); everything is tiny (~9.4k parameters), so the
// kernels favour simplicity: a CTA handles 32 samples with all weights in
// shared memory, and parameter gradients are summed with atomics.
//
// Parameter layout (floats): W1[64][D], b1[64], W2[64][64], b2[64],
// W3[64][64], b3[64], w4[64], b4.   y = w4 . g(W3 g(W2 g(W1 x + b1) + b2)
// + b3) + b4 with g(z) = z (1 + erf(z / sqrt 2)) / 2.
#include <cmath>
#include "common.cuh"

namespace gb {
namespace {

constexpr int H = 64;
constexpr int S = 32;      // samples per CTA
constexpr int NTM = 256;   // threads per CTA

__host__ __device__ inline int64_t pcount(int D) { return int64_t(H) * D + H + 2 * (int64_t(H) * H + H) + H + 1; }

__device__ __forceinline__ float gelu(float z) { return 0.5f * z * (1.0f + erff(z * 0.70710678118654752f)); }
__device__ __forceinline__ float gelu_d(float z)
{
    return 0.5f * (1.0f + erff(z * 0.70710678118654752f)) + z * expf(-0.5f * z * z) * 0.39894228040143268f;
}

// z[s][j] = b[j] + sum_k W[j][k] in[s][k]  for s < ns, j < H
__device__ void dense(const float *W, const float *b, const float *in, int kin, int ldin, float *z, int ns)
{
    for (int idx = threadIdx.x; idx < ns * H; idx += NTM) {
        const int s = idx / H, j = idx % H;
        float acc = b[j];
        for (int k = 0; k < kin; k++) acc = fmaf(W[j * kin + k], in[s * ldin + k], acc);
        z[s * H + j] = acc;
    }
}

__global__ void __launch_bounds__(NTM)
mlp_forward_kernel(const float *__restrict__ P, int D, const float *__restrict__ X, int64_t n, float *__restrict__ Y,
                   float *__restrict__ Z)
{
    extern __shared__ float sm[];
    const int64_t np = pcount(D);
    float *w = sm;
    float *x = w + np;           // S x D
    float *a = x + S * D;        // S x H (activations)
    float *z = a + S * H;        // S x H (pre-activations)
    for (int64_t i = threadIdx.x; i < np; i += NTM) w[i] = P[i];
    const int64_t s0 = int64_t(blockIdx.x) * S;
    const int ns = int((n - s0) < S ? (n - s0) : S);
    for (int i = threadIdx.x; i < ns * D; i += NTM) x[i] = X[s0 * D + i];
    __syncthreads();
    const float *W1 = w, *b1 = W1 + H * D, *W2 = b1 + H, *b2 = W2 + H * H, *W3 = b2 + H, *b3 = W3 + H * H;
    const float *w4 = b3 + H, *b4 = w4 + H;
    const float *Wl[3] = {W1, W2, W3}, *bl[3] = {b1, b2, b3};
    for (int l = 0; l < 3; l++) {
        dense(Wl[l], bl[l], l == 0 ? x : a, l == 0 ? D : H, l == 0 ? D : H, z, ns);
        __syncthreads();
        for (int idx = threadIdx.x; idx < ns * H; idx += NTM) {
            a[idx] = gelu(z[idx]);
            if (Z) Z[(s0 + idx / H) * 3 * H + l * H + idx % H] = z[idx];
        }
        __syncthreads();
    }
    // y = w4 . a + b4, one warp per sample
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int s = warp; s < ns; s += NTM / 32) {
        float acc = w4[lane] * a[s * H + lane] + w4[lane + 32] * a[s * H + lane + 32];
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if (lane == 0) Y[s0 + s] = acc + b4[0];
    }
}

// Per-sample backward with gradient accumulation into G (atomics).
__global__ void __launch_bounds__(NTM)
mlp_backward_kernel(const float *__restrict__ P, int D, const float *__restrict__ X, const float *__restrict__ Z,
                    const float *__restrict__ dY, int64_t n, float *__restrict__ G)
{
    extern __shared__ float sm[];
    const int64_t np = pcount(D);
    float *w = sm;
    float *x = w + np;               // S x D
    float *z = x + S * D;            // S x 3H
    float *d = z + S * 3 * H;        // S x H: current dZ
    float *t = d + S * H;            // S x H: scratch
    for (int64_t i = threadIdx.x; i < np; i += NTM) w[i] = P[i];
    const int64_t s0 = int64_t(blockIdx.x) * S;
    const int ns = int((n - s0) < S ? (n - s0) : S);
    for (int i = threadIdx.x; i < ns * D; i += NTM) x[i] = X[s0 * D + i];
    for (int i = threadIdx.x; i < ns * 3 * H; i += NTM) z[i] = Z[s0 * 3 * H + i];
    __syncthreads();
    const float *W1 = w, *b1 = W1 + H * D, *W2 = b1 + H, *b2 = W2 + H * H, *W3 = b2 + H, *b3 = W3 + H * H;
    const float *w4 = b3 + H;
    (void)b1; (void)b2; (void)b3;
    float *gW1 = G, *gb1 = gW1 + H * D, *gW2 = gb1 + H, *gb2 = gW2 + H * H, *gW3 = gb2 + H, *gb3 = gW3 + H * H;
    float *gw4 = gb3 + H, *gb4 = gw4 + H;
    auto Zl = [&](int s, int l, int j) { return z[s * 3 * H + l * H + j]; };

    // output layer: dY -> gw4, gb4; dZ3 = dY w4 g'(z3)
    for (int j = threadIdx.x; j < H; j += NTM) {
        float acc = 0.f;
        for (int s = 0; s < ns; s++) acc += dY[s0 + s] * gelu(Zl(s, 2, j));
        atomicAdd(&gw4[j], acc);
    }
    if (threadIdx.x == 0) {
        float acc = 0.f;
        for (int s = 0; s < ns; s++) acc += dY[s0 + s];
        atomicAdd(gb4, acc);
    }
    for (int idx = threadIdx.x; idx < ns * H; idx += NTM) {
        const int s = idx / H, j = idx % H;
        d[idx] = dY[s0 + s] * w4[j] * gelu_d(Zl(s, 2, j));
    }
    __syncthreads();
    // layers 3, 2, 1
    const float *Wl[3] = {W1, W2, W3};
    float *gWl[3] = {gW1, gW2, gW3}, *gbl[3] = {gb1, gb2, gb3};
    for (int l = 2; l >= 0; l--) {
        const int kin = l == 0 ? D : H;
        // grads: gW[j][k] += sum_s d[s][j] in[s][k], gb[j] += sum_s d[s][j]
        for (int idx = threadIdx.x; idx < H * kin; idx += NTM) {
            const int j = idx / kin, k = idx % kin;
            float acc = 0.f;
            for (int s = 0; s < ns; s++) {
                const float in = l == 0 ? x[s * D + k] : gelu(Zl(s, l - 1, k));
                acc = fmaf(d[s * H + j], in, acc);
            }
            atomicAdd(&gWl[l][idx], acc);
        }
        for (int j = threadIdx.x; j < H; j += NTM) {
            float acc = 0.f;
            for (int s = 0; s < ns; s++) acc += d[s * H + j];
            atomicAdd(&gbl[l][j], acc);
        }
        if (l == 0) break;
        // d_prev[s][k] = g'(z_{l-1}[s][k]) sum_j W_l[j][k] d[s][j]
        for (int idx = threadIdx.x; idx < ns * H; idx += NTM) {
            const int s = idx / H, k = idx % H;
            float acc = 0.f;
            for (int j = 0; j < H; j++) acc = fmaf(Wl[l][j * H + k], d[s * H + j], acc);
            t[idx] = acc * gelu_d(Zl(s, l - 1, k));
        }
        __syncthreads();
        for (int idx = threadIdx.x; idx < ns * H; idx += NTM) d[idx] = t[idx];
        __syncthreads();
    }
}

// dY = 2 (Y - T) / n, loss += sum (Y - T)^2 / n
__global__ void mlp_loss_kernel(const float *Y, const float *T, int64_t n, float *dY, float *loss)
{
    float acc = 0.f;
    for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x) {
        const float e = Y[i] - T[i];
        dY[i] = 2.f * e / float(n);
        acc += e * e / float(n);
    }
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0 && loss) atomicAdd(loss, acc);
}

__global__ void mlp_adam_kernel(float *P, const float *G, float *M, float *V, int64_t np, float lr, float b1,
                                float b2, float eps, float c1, float c2)
{
    for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < np; i += int64_t(gridDim.x) * blockDim.x) {
        const float g = G[i];
        const float m = b1 * M[i] + (1.f - b1) * g;
        const float v = b2 * V[i] + (1.f - b2) * g * g;
        M[i] = m;
        V[i] = v;
        P[i] -= lr * (m / c1) / (sqrtf(v / c2) + eps);
    }
}

size_t fwd_smem(int D) { return sizeof(float) * size_t(pcount(D) + S * D + 2 * S * H); }
size_t bwd_smem(int D) { return sizeof(float) * size_t(pcount(D) + S * D + 3 * S * H + 2 * S * H); }

int set_attrs(int D)
{
    // the limit depends on the input width D: set per call (cheap next to
    // the kernels, and correct on whichever device is current)
    GB_CUDA(cudaFuncSetAttribute(mlp_forward_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)fwd_smem(D)));
    GB_CUDA(cudaFuncSetAttribute(mlp_backward_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bwd_smem(D)));
    return 0;
}

}  // namespace

int mlp_forward(const float *P, int D, const float *X, int64_t n, float *Y, float *Z, cudaStream_t s)
{
    if (n <= 0) return 0;
    GB_TRY(set_attrs(D));
    const int64_t grid = (n + S - 1) / S;
    LaunchScope ls(KK_MLP, s, 2.0 * n * (double(H) * D + 2.0 * H * H + H), 4.0 * n * (D + 1));
    mlp_forward_kernel<<<(unsigned)grid, NTM, fwd_smem(D), s>>>(P, D, X, n, Y, Z);
    return check(cudaGetLastError());
}

}  // namespace gb

extern "C" {

int64_t gb_mlp_param_count(int in_dim) { return in_dim > 0 ? gb::pcount(in_dim) : -1; }

int gb_mlp_forward(const float *params, int in_dim, const float *X, int64_t n, float *Y, float *Z, void *stream)
{
    if (!params) return -1;
    if (in_dim < 1 || in_dim > 64) return -2;
    if (!X && n > 0) return -3;
    if (n < 0) return -4;
    if (!Y && n > 0) return -5;
    return gb::mlp_forward(params, in_dim, X, n, Y, Z, static_cast<cudaStream_t>(stream));
}

int gb_mlp_backward(const float *params, int in_dim, const float *X, const float *Z, const float *dY, int64_t n,
                    float *grads, void *stream)
{
    if (!params) return -1;
    if (in_dim < 1 || in_dim > 64) return -2;
    if (!X && n > 0) return -3;
    if (!Z && n > 0) return -4;
    if (!dY && n > 0) return -5;
    if (n < 0) return -6;
    if (!grads) return -7;
    if (n == 0) return 0;
    GB_TRY(gb::set_attrs(in_dim));
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int64_t grid = (n + gb::S - 1) / gb::S;
    gb::LaunchScope ls(gb::KK_MLP, s, 4.0 * n * gb::pcount(in_dim), 4.0 * n * (in_dim + 3 * gb::H + 1));
    gb::mlp_backward_kernel<<<(unsigned)grid, gb::NTM, gb::bwd_smem(in_dim), s>>>(params, in_dim, X, Z, dY, n, grads);
    return gb::check(cudaGetLastError());
}

int gb_mlp_loss(const float *Y, const float *T, int64_t n, float *dY, float *loss, void *stream)
{
    if (n < 0) return -3;
    if (n == 0) return 0;
    if (!Y) return -1;
    if (!T) return -2;
    if (!dY) return -4;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    gb::LaunchScope ls(gb::KK_MLP, s, 3.0 * n, 12.0 * n);
    gb::mlp_loss_kernel<<<(unsigned)((n + 255) / 256 < 1024 ? (n + 255) / 256 : 1024), 256, 0, s>>>(Y, T, n, dY, loss);
    return gb::check(cudaGetLastError());
}

int gb_mlp_adam(float *params, const float *grads, float *m, float *v, int64_t np, float lr, float beta1, float beta2,
                float eps, int step, void *stream)
{
    if (!params || !grads || !m || !v) return -1;
    if (np < 0) return -5;
    if (step < 1) return -10;
    if (np == 0) return 0;
    const float c1 = 1.f - std::pow(beta1, float(step)), c2 = 1.f - std::pow(beta2, float(step));
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    gb::LaunchScope ls(gb::KK_MLP, s, 10.0 * np, 20.0 * np);
    gb::mlp_adam_kernel<<<(unsigned)((np + 255) / 256), 256, 0, s>>>(params, grads, m, v, np, lr, beta1, beta2, eps, c1,
                                                                     c2);
    return gb::check(cudaGetLastError());
}

}  // extern "C"
